// Host-side set-up of the assembly data: the block-CSR pattern of K (one 3x3 block per pair
// of nodes that share an element), a conflict-free element colouring, and the element-to-
// block slot map that replaces the paper's triplet -> COO -> CSR assembly (App. E,
// Algorithm gpu_chunked_assembly): slot[e][a][b] is the index of block (conn[e][a],
// conn[e][b]); bit 31 marks the first launch (in launch order) that writes the block, which
// stores instead of adding, so K needs no clearing pass.  Also here: the cut of the rows into
// the chunks that the streamed CG copies into shared memory.
#include "pattern.h"

#include <algorithm>
#include <cstring>
#include <thread>

namespace hfe {

static void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < 4096 || nt == 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min<int64_t>(n, b + chunk);
    if (b >= e) break;
    th.emplace_back(f, b, e);
  }
  for (auto& x : th) x.join();
}

bool build_pattern(int64_t n_nodes, int64_t n_el, const int32_t* conn, const SlabPlan& plan, Pattern& P,
                   std::string& err) {
  for (int64_t i = 0; i < n_el * 8; ++i) {
    if (conn[i] < 0 || conn[i] >= n_nodes) {
      err = "conn[" + std::to_string(i) + "] out of range";
      return false;
    }
  }
  for (int64_t e = 0; e < n_el; ++e)
    for (int a = 0; a < 8; ++a)
      for (int b = a + 1; b < 8; ++b)
        if (conn[e * 8 + a] == conn[e * 8 + b]) {
          err = "element " + std::to_string(e) + " repeats a node";
          return false;
        }
  // node -> elements incidence
  std::vector<int64_t> nptr(n_nodes + 1, 0);
  for (int64_t i = 0; i < n_el * 8; ++i) nptr[conn[i] + 1]++;
  for (int64_t n = 0; n < n_nodes; ++n) nptr[n + 1] += nptr[n];
  for (int64_t n = 0; n < n_nodes; ++n) {
    if (nptr[n + 1] == nptr[n]) {
      err = "node " + std::to_string(n) + " belongs to no element";
      return false;
    }
  }
  std::vector<int32_t> nel(n_el * 8);
  {
    std::vector<int64_t> fill(nptr.begin(), nptr.end() - 1);
    for (int64_t e = 0; e < n_el; ++e)
      for (int a = 0; a < 8; ++a) nel[fill[conn[e * 8 + a]]++] = (int32_t)e;
  }
  // rows: sorted unique neighbour nodes
  std::vector<int64_t> cnt(n_nodes, 0);
  std::vector<std::vector<int32_t>> rows(n_nodes);
  parallel_for(n_nodes, [&](int64_t b, int64_t e) {
    std::vector<int32_t> buf;
    for (int64_t n = b; n < e; ++n) {
      buf.clear();
      for (int64_t k = nptr[n]; k < nptr[n + 1]; ++k) {
        const int32_t* c = conn + (int64_t)nel[k] * 8;
        buf.insert(buf.end(), c, c + 8);
      }
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
      rows[n] = buf;
    }
  });
  P.rowptr.assign(n_nodes + 1, 0);
  for (int64_t n = 0; n < n_nodes; ++n) P.rowptr[n + 1] = P.rowptr[n] + (int64_t)rows[n].size();
  P.n_blocks = P.rowptr[n_nodes];
  if (P.n_blocks >= (int64_t)0x7fffffff) {
    err = "more than 2^31 - 1 blocks";
    return false;
  }
  P.cols.resize(P.n_blocks);
  P.diag_slot.resize(n_nodes);
  parallel_for(n_nodes, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e; ++n) {
      std::copy(rows[n].begin(), rows[n].end(), P.cols.begin() + P.rowptr[n]);
      auto it = std::lower_bound(rows[n].begin(), rows[n].end(), (int32_t)n);
      P.diag_slot[n] = P.rowptr[n] + (it - rows[n].begin());
      std::vector<int32_t>().swap(rows[n]);
    }
  });
  // greedy colouring: the smallest colour not used by an element sharing a node
  std::vector<int8_t> color(n_el, -1);
  int ncol = 0;
  for (int64_t e = 0; e < n_el; ++e) {
    uint64_t used = 0;
    for (int a = 0; a < 8; ++a) {
      int32_t n = conn[e * 8 + a];
      for (int64_t k = nptr[n]; k < nptr[n + 1]; ++k) {
        int8_t c = color[nel[k]];
        if (c >= 0) used |= (1ull << c);
      }
    }
    int c = 0;
    while (c < 64 && (used >> c & 1ull)) ++c;
    if (c >= 64) {
      err = "element colouring needs more than 64 colours";
      return false;
    }
    color[e] = (int8_t)c;
    ncol = std::max(ncol, c + 1);
  }
  P.n_colors = ncol;
  // launch order.  A launch is one colour, so its elements share no node; the launches are
  // ordered by slab, then colour: the eight or so colours of a slab add into a band of K
  // rows small enough to stay in L2 between them, instead of each colour sweeping all of K.
  // The slab of an element is that of the first K block of its lowest-numbered node's row.
  std::vector<int64_t> slab(n_el, 0);
  P.n_slabs = 1;
  P.slab_blocks = 0;
  if (plan.max_blocks > 0 && n_el > 0) {
    std::vector<int64_t> first(n_el);
    for (int64_t e = 0; e < n_el; ++e) {
      int32_t lo = conn[e * 8];
      for (int a = 1; a < 8; ++a) lo = std::min(lo, conn[e * 8 + a]);
      first[e] = P.rowptr[lo];
    }
    const int64_t lo_b = std::max<int64_t>(1, std::min(plan.min_blocks, plan.max_blocks));
    const int64_t hi_b = std::max<int64_t>(lo_b, plan.max_blocks);
    const int64_t res = std::max<int64_t>(1, plan.resident_ctas), epc = std::max<int64_t>(1, plan.el_per_cta);
    int64_t best_sb = hi_b, best_w = -1;
    const int n_cand = hi_b > lo_b ? 32 : 1;
    std::vector<int64_t> cnt;
    for (int k = n_cand - 1; k >= 0; --k) {   // largest first: a tie keeps the larger size
      const int64_t sb = n_cand == 1 ? hi_b : lo_b + (hi_b - lo_b) * k / 31;
      const int64_t ns = P.n_blocks / sb + 1;
      cnt.assign(ns * ncol, 0);
      for (int64_t e = 0; e < n_el; ++e) cnt[first[e] / sb * ncol + color[e]]++;
      int64_t w = 0;
      for (int64_t c : cnt) w += ((c + epc - 1) / epc + res - 1) / res;
      if (best_w < 0 || w < best_w) {
        best_w = w;
        best_sb = sb;
      }
    }
    P.slab_blocks = best_sb;
    for (int64_t e = 0; e < n_el; ++e) {
      slab[e] = first[e] / best_sb;
      P.n_slabs = std::max(P.n_slabs, slab[e] + 1);
    }
  }
  // colour order, then a stable counting sort by slab
  std::vector<int64_t> coff(ncol + 1, 0);
  for (int64_t e = 0; e < n_el; ++e) coff[color[e] + 1]++;
  for (int c = 0; c < ncol; ++c) coff[c + 1] += coff[c];
  std::vector<int32_t> by_colour(n_el);
  for (int64_t e = 0; e < n_el; ++e) by_colour[coff[color[e]]++] = (int32_t)e;
  std::vector<int64_t> soff(P.n_slabs + 1, 0);
  for (int64_t e = 0; e < n_el; ++e) soff[slab[e] + 1]++;
  for (int64_t g = 0; g < P.n_slabs; ++g) soff[g + 1] += soff[g];
  P.elems.resize(n_el);
  for (int64_t i = 0; i < n_el; ++i) {
    const int32_t e = by_colour[i];
    P.elems[soff[slab[e]]++] = e;
  }
  P.launch_off.assign(1, 0);
  for (int64_t i = 1; i < n_el; ++i) {
    const int32_t e0 = P.elems[i - 1], e1 = P.elems[i];
    if (slab[e0] != slab[e1] || color[e0] != color[e1]) P.launch_off.push_back(i);
  }
  if (n_el > 0) P.launch_off.push_back(n_el);
  // slot map
  P.slot.resize(n_el * 64);
  parallel_for(n_el, [&](int64_t b, int64_t e_end) {
    for (int64_t e = b; e < e_end; ++e) {
      for (int a = 0; a < 8; ++a) {
        int32_t r = conn[e * 8 + a];
        const int32_t* c0 = P.cols.data() + P.rowptr[r];
        const int32_t* c1 = P.cols.data() + P.rowptr[r + 1];
        for (int bb = 0; bb < 8; ++bb) {
          const int32_t* it = std::lower_bound(c0, c1, conn[e * 8 + bb]);
          P.slot[e * 64 + a * 8 + bb] = (int32_t)(P.rowptr[r] + (it - c0));
        }
      }
    }
  });
  // first-writer flags in launch order (one writer per block per launch)
  std::vector<uint8_t> seen(P.n_blocks, 0);
  for (int64_t i = 0; i < n_el; ++i) {
    int64_t e = P.elems[i];
    for (int k = 0; k < 64; ++k) {
      int32_t s = P.slot[e * 64 + k];
      if (!seen[s]) {
        seen[s] = 1;
        P.slot[e * 64 + k] = (int32_t)((uint32_t)s | 0x80000000u);
      }
    }
  }
  return true;
}

void stream_chunks(const int64_t* rowptr, int64_t n_nodes, int max_rows, int max_blocks, std::vector<int32_t>& out) {
  out.clear();
  out.push_back(0);
  int64_t r = 0;
  while (r < n_nodes) {
    const int64_t r0 = r;
    while (r < n_nodes && r - r0 < max_rows && rowptr[r + 1] - rowptr[r0] <= max_blocks) ++r;
    if (r == r0) {   // a row longer than a chunk: no streamed SpMV for this pattern
      out.clear();
      return;
    }
    out.push_back((int32_t)r);
  }
}

}  // namespace hfe
