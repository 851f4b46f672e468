// Internal declarations shared by the libmg translation units (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mg.h"

namespace mg {

constexpr int kSlotAlign = 32;

inline int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// Host tables of one spacetree level (see the level layout in mg.h).
struct HostLevel {
  int level = 0, dim = 0;
  int n = 0;        // cells per axis, 3^level
  int B = 0;        // brick edge
  int S = 0;        // slots per brick
  int m = 0;        // brick depth
  int nb_axis = 0;  // brick roots per axis, 3^(level-m)
  double h = 0.0;
  int64_t n_bricks = 0, n_slots = 0, n_dofs = 0, n_cells = 0, n_hanging = 0, slot_offset = 0;
  std::vector<int32_t> brick_roots;  // n_bricks*d
  std::vector<int32_t> brick_rank;   // nb_axis^d, -1 if unallocated
  std::vector<int32_t> brick_nbr;    // n_bricks*3^d
  std::vector<uint8_t> vflags, cflags;
  std::vector<int32_t> hang_idx;     // n_slots*2^d
  std::vector<double> hang_w;
  // slot of an integer position, -1 if outside [0,n)^d or unallocated
  int64_t slot_of(const int* x) const;
  void coords_of(int64_t slot, int* x) const;  // -1s on padding slots
};

struct Grid {
  int dim = 0, L = 0;
  std::vector<std::vector<uint8_t>> cells, refined;  // per level, lexicographic (3^l)^d
  std::vector<HostLevel> levels;
  bool uniform = true;
};

// Peano coordinates of a level-`level` cell with curve index t (digit rule of Sect. 3 / App. A).
void peano_coords(int dim, int level, int64_t t, int* coords);

// Fills lv (flags, bricks, hanging map) for level l of g; defined in grid.cpp.
void build_level(const Grid& g, int l, HostLevel& lv);

void set_error(const std::string& msg);

}  // namespace mg
