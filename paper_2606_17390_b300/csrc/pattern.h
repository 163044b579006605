// Assembly pattern built on the host (internal).
#pragma once

#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

namespace hfe {

struct Pattern {
  std::vector<int64_t> rowptr;     // [n_nodes + 1]
  std::vector<int32_t> cols;       // [n_blocks]
  std::vector<int64_t> diag_slot;  // [n_nodes]
  std::vector<int32_t> slot;       // [n_el * 64], bit 31 = first writer
  std::vector<int32_t> elems;      // element ids in launch order
  std::vector<int64_t> launch_off; // [n_launches + 1]: the conflict-free ranges of elems
  int64_t n_blocks = 0;
  int64_t n_slabs = 1;
  int64_t slab_blocks = 0;         // the slab size chosen (0: one slab)
  int n_colors = 0;
};

// Launch order.  Elements are grouped by the slab of slab_blocks consecutive K blocks (in row
// order) that holds the first row they write, then by colour within a slab; one launch per
// non-empty (slab, colour).  max_blocks == 0: one slab (one launch per colour).  min_blocks ==
// max_blocks: that slab size.  Otherwise the size is chosen among the 32 sizes
// min + (max - min) k / 31, k = 0..31, as the one whose launches take the fewest waves of
// resident_ctas CTAs of el_per_cta elements (sum over launches of ceil(CTAs / resident_ctas)),
// the larger size on a tie: a launch's partial last wave is time the next launch's assembly
// waits for.
struct SlabPlan {
  int64_t min_blocks = 0, max_blocks = 0;
  int64_t resident_ctas = 1;
  int64_t el_per_cta = 16;
};

bool build_pattern(int64_t n_nodes, int64_t n_el, const int32_t* conn, const SlabPlan& plan, Pattern& P,
                   std::string& err);

// Row chunks of the streamed CG SpMV: greedy runs of consecutive rows, each of at most
// max_rows rows and max_blocks blocks (rowptr[end] - rowptr[start] <= max_blocks); out =
// [0, end_0, end_1, ..., n_nodes].  out is empty when a single row has more than max_blocks
// blocks (the CG then loads K directly).
void stream_chunks(const int64_t* rowptr, int64_t n_nodes, int max_rows, int max_blocks, std::vector<int32_t>& out);

}  // namespace hfe
