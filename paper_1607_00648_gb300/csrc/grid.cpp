// Host-side spacetree flattening (A1): k = 3 spacetree (Sect. 3) -> level arrays in
// Peano brick order with vertex flags, neighbour / hanging / injection tables.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace mg {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// Index -> coordinates of the Peano curve: the index has ternary digits t_1 t_2 ...
// (dim digits per level, axis 0 first, most significant first).  A digit of axis i
// becomes the coordinate digit t or 2 - t, the latter iff the digits seen so far on
// the other axes sum to an odd number (Peano's serpentine construction).
void peano_coords(int dim, int level, int64_t t, int* coords) {
  const int nd = dim * level;
  int digits[3 * 16];
  int64_t v = t;
  for (int p = nd - 1; p >= 0; --p) {
    digits[p] = static_cast<int>(v % 3);
    v /= 3;
  }
  int sums[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) coords[i] = 0;
  for (int p = 0; p < nd; ++p) {
    const int axis = p % dim;
    int other = 0;
    for (int j = 0; j < dim; ++j)
      if (j != axis) other += sums[j];
    const int a = (other & 1) ? 2 - digits[p] : digits[p];
    coords[axis] = coords[axis] * 3 + a;
    sums[axis] += digits[p];
  }
}

int64_t HostLevel::slot_of(const int* x) const {
  int r[3], l[3];
  for (int i = 0; i < dim; ++i) {
    if (x[i] < 0 || x[i] >= n) return -1;
    r[i] = x[i] / B;
    l[i] = x[i] % B;
  }
  int64_t ri = 0, li = 0;
  for (int i = dim - 1; i >= 0; --i) {
    ri = ri * nb_axis + r[i];
    li = li * B + l[i];
  }
  const int32_t rank = brick_rank[ri];
  if (rank < 0) return -1;
  return static_cast<int64_t>(rank) * S + li;
}

void HostLevel::coords_of(int64_t slot, int* x) const {
  const int64_t b = slot / S;
  int64_t k = slot % S;
  if (k >= static_cast<int64_t>(ipow(B, dim))) {
    for (int i = 0; i < dim; ++i) x[i] = -1;
    return;
  }
  for (int i = 0; i < dim; ++i) {
    x[i] = brick_roots[b * dim + i] * B + static_cast<int>(k % B);
    k /= B;
  }
}

static inline int64_t lex_index(const int* x, int n, int dim) {
  int64_t r = 0;
  for (int i = dim - 1; i >= 0; --i) r = r * n + x[i];
  return r;
}

void build_level(const Grid& g, int l, HostLevel& lv) {
  const int d = g.dim;
  lv.level = l;
  lv.dim = d;
  lv.n = ipow(3, l);
  lv.m = std::min(l, d == 2 ? 3 : 2);
  lv.B = ipow(3, lv.m);
  const int nloc = ipow(lv.B, d);
  lv.S = ((nloc + kSlotAlign - 1) / kSlotAlign) * kSlotAlign;
  lv.nb_axis = ipow(3, l - lv.m);
  lv.h = 1.0;
  for (int i = 0; i < l; ++i) lv.h /= 3.0;
  const std::vector<uint8_t>& cells = g.cells[l];
  const std::vector<uint8_t>& refd = g.refined[l];
  const int nbr_count = ipow(lv.nb_axis, d);

  // bricks that contain existing cells
  std::vector<uint8_t> has(nbr_count, 0);
  const int64_t ncell = static_cast<int64_t>(ipow(lv.n, d));
  int x[3], r[3];
  for (int64_t c = 0; c < ncell; ++c) {
    if (!cells[c]) continue;
    int64_t v = c;
    for (int i = 0; i < d; ++i) {
      x[i] = static_cast<int>(v % lv.n);
      v /= lv.n;
      r[i] = x[i] / lv.B;
    }
    has[lex_index(r, lv.nb_axis, d)] = 1;
  }
  // allocation: a brick is kept iff it or a brick at root offset -e, e in {0,1}^d, has cells
  std::vector<uint8_t> alloc(nbr_count, 0);
  for (int64_t ri = 0; ri < nbr_count; ++ri) {
    int64_t v = ri;
    for (int i = 0; i < d; ++i) {
      r[i] = static_cast<int>(v % lv.nb_axis);
      v /= lv.nb_axis;
    }
    for (int e = 0; e < (1 << d) && !alloc[ri]; ++e) {
      int q[3];
      bool ok = true;
      for (int i = 0; i < d; ++i) {
        q[i] = r[i] - ((e >> i) & 1);
        if (q[i] < 0) ok = false;
      }
      if (ok && has[lex_index(q, lv.nb_axis, d)]) alloc[ri] = 1;
    }
  }
  // Peano order of the allocated brick roots
  lv.brick_rank.assign(nbr_count, -1);
  lv.brick_roots.clear();
  int64_t nb = 0;
  for (int64_t t = 0; t < nbr_count; ++t) {
    peano_coords(d, l - lv.m, t, r);
    const int64_t ri = lex_index(r, lv.nb_axis, d);
    if (!alloc[ri]) continue;
    lv.brick_rank[ri] = static_cast<int32_t>(nb++);
    for (int i = 0; i < d; ++i) lv.brick_roots.push_back(r[i]);
  }
  lv.n_bricks = nb;
  lv.n_slots = nb * lv.S;

  // brick neighbour table
  const int n3 = ipow(3, d);
  lv.brick_nbr.assign(nb * n3, -1);
  for (int64_t b = 0; b < nb; ++b) {
    for (int k = 0; k < n3; ++k) {
      int q[3];
      bool ok = true;
      int kk = k;
      for (int i = 0; i < d; ++i) {
        q[i] = lv.brick_roots[b * d + i] + (kk % 3) - 1;
        kk /= 3;
        if (q[i] < 0 || q[i] >= lv.nb_axis) ok = false;
      }
      if (ok) lv.brick_nbr[b * n3 + k] = lv.brick_rank[lex_index(q, lv.nb_axis, d)];
    }
  }

  // vertex and cell flags (Sect. 3)
  lv.vflags.assign(lv.n_slots, 0);
  lv.cflags.assign(lv.n_slots, 0);
  lv.n_dofs = lv.n_cells = lv.n_hanging = 0;
  const int full = 1 << d;
  for (int64_t s = 0; s < lv.n_slots; ++s) {
    lv.coords_of(s, x);
    if (x[0] < 0) continue;
    const int64_t cidx = lex_index(x, lv.n, d);
    if (cells[cidx]) {
      lv.cflags[s] |= MG_C_EXISTS;
      ++lv.n_cells;
    }
    if (refd[cidx]) lv.cflags[s] |= MG_C_REFINED;
    int n_adj = 0, n_ref = 0;
    for (int e = 0; e < full; ++e) {
      int q[3];
      bool ok = true;
      for (int i = 0; i < d; ++i) {
        q[i] = x[i] - ((e >> i) & 1);
        if (q[i] < 0) ok = false;
      }
      if (!ok) continue;
      const int64_t qi = lex_index(q, lv.n, d);
      n_adj += cells[qi] ? 1 : 0;
      n_ref += refd[qi] ? 1 : 0;
    }
    if (n_adj == 0) continue;
    uint8_t f = MG_V_EXISTS;
    bool bnd = false;
    for (int i = 0; i < d; ++i)
      if (x[i] == 0) bnd = true;
    if (bnd) {
      f |= MG_V_BOUNDARY;
    } else if (n_adj < full) {
      f |= MG_V_HANGING;
      ++lv.n_hanging;
    } else {
      if (n_ref == full) f |= MG_V_REFINED;
      ++lv.n_dofs;
    }
    lv.vflags[s] = f;
  }
}

}  // namespace mg

using namespace mg;

extern "C" {

const char* mg_last_error(void) { return g_last_error.c_str(); }
const char* mg_version(void) { return "libmg 0.1 (sm_103a)"; }

mg_status mg_create_grid(int dim, int max_level, const uint8_t* const* refine_masks, mg_grid** out) {
  if (!out) {
    set_error("mg_create_grid: out is NULL");
    return MG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (dim != 2 && dim != 3) {
    set_error("mg_create_grid: dim must be 2 or 3");
    return MG_ERR_INVALID_ARG;
  }
  if (max_level < 1 || max_level > (dim == 2 ? 8 : 6)) {
    set_error("mg_create_grid: max_level out of range");
    return MG_ERR_INVALID_ARG;
  }
  try {
    Grid* g = new Grid();
    g->dim = dim;
    g->L = max_level;
    g->cells.resize(max_level + 1);
    g->refined.resize(max_level + 1);
    g->cells[0].assign(1, 1);
    for (int l = 0; l <= max_level; ++l) {
      const int n = ipow(3, l);
      const int64_t nc = static_cast<int64_t>(ipow(n, dim));
      std::vector<uint8_t>& rf = g->refined[l];
      rf.assign(nc, 0);
      if (l < max_level) {
        const uint8_t* mask = refine_masks ? refine_masks[l] : nullptr;
        for (int64_t c = 0; c < nc; ++c) {
          rf[c] = (g->cells[l][c] && (!mask || mask[c])) ? 1 : 0;
          if (g->cells[l][c] && !rf[c]) g->uniform = false;
        }
        // children of refined cells exist on level l+1
        const int nf = 3 * n;
        std::vector<uint8_t>& cf = g->cells[l + 1];
        cf.assign(static_cast<int64_t>(ipow(nf, dim)), 0);
        int x[3];
        for (int64_t c = 0; c < static_cast<int64_t>(cf.size()); ++c) {
          int64_t v = c;
          int64_t pc = 0, mul = 1;
          for (int i = 0; i < dim; ++i) {
            x[i] = static_cast<int>(v % nf);
            v /= nf;
            pc += (x[i] / 3) * mul;
            mul *= n;
          }
          cf[c] = rf[pc];
        }
      }
    }
    g->levels.resize(max_level + 1);
    int64_t off = 0;
    for (int l = 0; l <= max_level; ++l) {
      build_level(*g, l, g->levels[l]);
      g->levels[l].slot_offset = off;
      off += g->levels[l].n_slots;
    }
    // hanging maps need the coarser level
    for (int l = 1; l <= max_level; ++l) {
      HostLevel& lv = g->levels[l];
      const HostLevel& co = g->levels[l - 1];
      const int full = 1 << dim;
      lv.hang_idx.assign(lv.n_slots * full, -1);
      lv.hang_w.assign(lv.n_slots * full, 0.0);
      int x[3];
      for (int64_t s = 0; s < lv.n_slots; ++s) {
        if (!(lv.vflags[s] & MG_V_HANGING)) continue;
        lv.coords_of(s, x);
        for (int e = 0; e < full; ++e) {
          double w = 1.0;
          int X[3];
          for (int i = 0; i < dim; ++i) {
            const int ei = (e >> i) & 1;
            const int ri = x[i] % 3;
            const double f = ei ? ri / 3.0 : (3 - ri) / 3.0;
            w = (i == 0) ? f : w * f;
            X[i] = x[i] / 3 + ei;
          }
          if (w == 0.0) continue;
          const int64_t cs = co.slot_of(X);
          if (cs < 0) continue;
          lv.hang_idx[s * full + e] = static_cast<int32_t>(cs);
          lv.hang_w[s * full + e] = w;
        }
      }
    }
    *out = reinterpret_cast<mg_grid*>(g);
  } catch (const std::bad_alloc&) {
    set_error("mg_create_grid: out of host memory");
    return MG_ERR_OOM;
  }
  return MG_OK;
}

mg_status mg_grid_info(const mg_grid* grid, int level, mg_level_info* info) {
  const Grid* g = reinterpret_cast<const Grid*>(grid);
  if (!g || !info || level < 0 || level > g->L) {
    set_error("mg_grid_info: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  const HostLevel& lv = g->levels[level];
  info->level = level;
  info->dim = g->dim;
  info->brick_edge = lv.B;
  info->slots_per_brick = lv.S;
  info->n_bricks = lv.n_bricks;
  info->n_slots = lv.n_slots;
  info->n_dofs = lv.n_dofs;
  info->n_cells = lv.n_cells;
  info->n_hanging = lv.n_hanging;
  info->slot_offset = lv.slot_offset;
  info->h = lv.h;
  return MG_OK;
}

mg_status mg_grid_tables(const mg_grid* grid, int level, int32_t* coords, uint8_t* vflags, uint8_t* cflags,
                         int32_t* nbr, int32_t* cell_vertices, int32_t* hang_idx, double* hang_w,
                         int32_t* parent, int32_t* child, int32_t* brick_roots, int32_t* brick_nbr) {
  const Grid* g = reinterpret_cast<const Grid*>(grid);
  if (!g || level < 0 || level > g->L) {
    set_error("mg_grid_tables: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  const HostLevel& lv = g->levels[level];
  const int d = g->dim;
  const int n3 = ipow(3, d), full = 1 << d;
  int x[3], y[3];
  for (int64_t s = 0; s < lv.n_slots; ++s) {
    lv.coords_of(s, x);
    const bool valid = x[0] >= 0;
    if (coords)
      for (int i = 0; i < d; ++i) coords[s * d + i] = x[i];
    if (nbr) {
      for (int k = 0; k < n3; ++k) {
        int64_t v = -1;
        if (valid) {
          int kk = k;
          for (int i = 0; i < d; ++i) {
            y[i] = x[i] + (kk % 3) - 1;
            kk /= 3;
          }
          v = lv.slot_of(y);
        }
        nbr[s * n3 + k] = static_cast<int32_t>(v);
      }
    }
    if (cell_vertices) {
      for (int e = 0; e < full; ++e) {
        int64_t v = -1;
        if (valid) {
          for (int i = 0; i < d; ++i) y[i] = x[i] + ((e >> i) & 1);
          v = lv.slot_of(y);
        }
        cell_vertices[s * full + e] = static_cast<int32_t>(v);
      }
    }
    if (parent) {
      int64_t v = -1;
      if (valid && level > 0) {
        bool c = true;
        for (int i = 0; i < d; ++i) {
          if (x[i] % 3) c = false;
          y[i] = x[i] / 3;
        }
        if (c) v = g->levels[level - 1].slot_of(y);
      }
      parent[s] = static_cast<int32_t>(v);
    }
    if (child) {
      int64_t v = -1;
      if (valid && level < g->L) {
        for (int i = 0; i < d; ++i) y[i] = 3 * x[i];
        v = g->levels[level + 1].slot_of(y);
      }
      child[s] = static_cast<int32_t>(v);
    }
  }
  if (vflags) std::memcpy(vflags, lv.vflags.data(), lv.n_slots);
  if (cflags) std::memcpy(cflags, lv.cflags.data(), lv.n_slots);
  if (hang_idx) {
    if (level == 0)
      std::fill(hang_idx, hang_idx + lv.n_slots * full, -1);
    else
      std::memcpy(hang_idx, lv.hang_idx.data(), lv.hang_idx.size() * sizeof(int32_t));
  }
  if (hang_w) {
    if (level == 0)
      std::fill(hang_w, hang_w + lv.n_slots * full, 0.0);
    else
      std::memcpy(hang_w, lv.hang_w.data(), lv.hang_w.size() * sizeof(double));
  }
  if (brick_roots) std::memcpy(brick_roots, lv.brick_roots.data(), lv.brick_roots.size() * sizeof(int32_t));
  if (brick_nbr) std::memcpy(brick_nbr, lv.brick_nbr.data(), lv.brick_nbr.size() * sizeof(int32_t));
  return MG_OK;
}

void mg_destroy_grid(mg_grid* grid) { delete reinterpret_cast<Grid*>(grid); }

}  // extern "C"
