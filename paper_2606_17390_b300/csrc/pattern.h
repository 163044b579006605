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
  std::vector<int32_t> elems;      // colour-sorted element ids
  std::vector<int64_t> color_off;  // [n_colors + 1]
  int64_t n_blocks = 0;
  int n_colors = 0;
};

bool build_pattern(int64_t n_nodes, int64_t n_el, const int32_t* conn, Pattern& P, std::string& err);

}  // namespace hfe
