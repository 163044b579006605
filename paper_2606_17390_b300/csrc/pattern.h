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
  int n_colors = 0;
};

// slab_blocks > 0: elements are grouped by the slab of slab_blocks consecutive K blocks (in
// row order) that holds the first row they write, and by colour within a slab; one launch
// per non-empty (slab, colour).  0: one slab, one launch per colour.
bool build_pattern(int64_t n_nodes, int64_t n_el, const int32_t* conn, int64_t slab_blocks, Pattern& P,
                   std::string& err);

}  // namespace hfe
