// Sector assignment, sector-sorted reordering and Verlet neighbour lists.
//
// Sectoring follows Sec. 5.1 of arXiv 1801.10233: the box is cut into an
// even number of sectors per edge, each at least (exchange cutoff + skin)
// wide, and sector (sx,sy,sz) gets colour (sx&1) + 2(sy&1) + 4(sz&1).  Atoms
// are stored sorted by (colour, sector, atom id), which is also the order of
// the sequential sweep of Eq. spin_ST_sectoring.  Sectors are assigned when
// the lists are rebuilt (not every step): each atom then moves at most skin/2
// before the next assignment, so same-colour sectors stay out of exchange
// range.
//
// Every kernel here runs only while ctrl->need_rebuild is set, so the whole
// sequence can sit in the step's launch sequence (and in a CUDA graph) and
// costs one early-exit per kernel when no rebuild is due.
#include <algorithm>

#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_pair.cuh"

namespace {

__global__ void k_rb_zero(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.nsec; q += gridDim.x * blockDim.x) {
    d.sec_count[q] = 0;
    d.sec_fill[q] = 0;
  }
}

// Wrap positions into their replica's box and find each atom's sector rank.
__global__ void k_rb_assign(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
    const SlRep& R = d.reps[d.arep[k]];
    double4_32a p = d.r[k];
    p.x = sl_wrap(p.x, R.box[0]);
    p.y = sl_wrap(p.y, R.box[1]);
    p.z = sl_wrap(p.z, R.box[2]);
    d.r[k] = p;
    int sx = sl_sector_coord(p.x, R.edge[0], R.nx);
    int sy = sl_sector_coord(p.y, R.edge[1], R.ny);
    int sz = sl_sector_coord(p.z, R.edge[2], R.nz);
    int q = sl_sector_rank(d, R, sx, sy, sz);
    d.tsecq[k] = q;
    atomicAdd(&d.sec_count[q], 1);
  }
}

// Exclusive scan of the sector counts (one block; rebuild-only).
__global__ void k_rb_scan(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  __shared__ int part[1024];
  int t = threadIdx.x, nt = blockDim.x;
  int chunk = (d.nsec + nt - 1) / nt;
  int a = t * chunk, b = min(d.nsec, a + chunk);
  int sum = 0;
  for (int q = a; q < b; ++q) sum += d.sec_count[q];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int u = 0; u < nt; ++u) { int x = part[u]; part[u] = acc; acc += x; }
  }
  __syncthreads();
  int acc = part[t];
  for (int q = a; q < b; ++q) { d.sec_start[q] = acc; acc += d.sec_count[q]; }
  if (t == nt - 1) d.sec_start[d.nsec] = acc;
}

__global__ void k_rb_scatter(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
    int q = d.tsecq[k];
    int pos = d.sec_start[q] + atomicAdd(&d.sec_fill[q], 1);
    d.src[pos] = k;
  }
}

// Order each sector's atoms by atom id (insertion sort; sectors hold ~10).
__global__ void k_rb_sort(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.nsec; q += gridDim.x * blockDim.x) {
    int a = d.sec_start[q], b = d.sec_start[q + 1];
    for (int x = a + 1; x < b; ++x) {
      int v = d.src[x];
      int id = d.perm[v];
      int y = x - 1;
      while (y >= a && d.perm[d.src[y]] > id) { d.src[y + 1] = d.src[y]; --y; }
      d.src[y + 1] = v;
    }
  }
}

__global__ void k_rb_gather(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
    int o = d.src[k];
    d.tr[k] = d.r[o];
    d.tv[k] = d.v[o];
    d.ts[k] = d.s[o];
    d.tF[k] = d.F[o];
    d.tperm[k] = d.perm[o];
    d.tarep[k] = d.arep[o];
    d.secq[k] = d.tsecq[o];
  }
}

__global__ void k_rb_copyback(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
    double4_32a p = d.tr[k];
    d.r[k] = p;
    d.rbx[k] = fx_pos(p);
    d.v[k] = d.tv[k];
    d.s[k] = d.ts[k];
    d.F[k] = d.tF[k];
    int id = d.tperm[k];
    d.perm[k] = id;
    d.rank[id] = k;
    d.arep[k] = d.tarep[k];
  }
}

// Full Verlet lists (both directions) from the sectors around each atom:
// exchange list r < ex_rc + skin, Morse list r < morse_rc + skin, both
// neighbour-major.  Neighbour order is the fixed loop order, so rebuilds are
// deterministic.  Each exchange list is reordered stably so that neighbours
// in the atom's own sector come first (exin[i] of them): the sweep sums the
// other sectors' field in parallel and only these in sequence.  The other
// neighbours follow grouped by their sector's colour (exc[i] holds the group
// starts), so a colour pass reads just the colour it needs.  The Morse
// list starts with the exchange list (same order) followed by the
// Morse-only neighbours, so the force loop takes the magneto-elastic branch
// only for its first exn[i] entries.  Requires morse_rc >= ex_rc.  The
// Morse-only neighbours come in three groups, each in loop order: those
// closer than morse_rc - skin at the build, which stay inside the cutoff
// until the next rebuild (no atom moves more than skin/2 before one); then
// those inside morse_rc at the build; then those outside it.  mnc[i] marks
// the end of the first group.  In a lattice every atom of a warp reaches the
// same group at the same entry, so the force loop's cutoff test takes the
// same branch across the warp.
// Membership uses float distances from the fixed-point positions with a
// relative margin of 1e-4 on r^2 (far above their rounding): a list may hold a pair
// marginally outside its radius, which is harmless because every kernel
// applies the exact cutoff to the pairs it reads.
__global__ void k_rb_nbr(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += gridDim.x * blockDim.x) {
    const SlRep& R = d.reps[d.arep[i]];
    const p3 pi = load_pos(d, i);
    const box3 B = load_box(d, R);
    const float lm2 = (float)d.list_m2 * 1.0001f, le2 = (float)d.list_ex2 * 1.0001f;
    const float lc2 = (float)d.sure_m2 * 0.9999f;     // (morse_rc - skin)^2, margin inward
    int sx, sy, sz;
    sl_sector_coords(d, R, d.secq[i], sx, sy, sz);
    int lox = (2 * R.mx + 1 >= R.nx) ? 0 : -R.mx, hix = (2 * R.mx + 1 >= R.nx) ? R.nx - 1 : R.mx;
    int loy = (2 * R.my + 1 >= R.ny) ? 0 : -R.my, hiy = (2 * R.my + 1 >= R.ny) ? R.ny - 1 : R.my;
    int loz = (2 * R.mz + 1 >= R.nz) ? 0 : -R.mz, hiz = (2 * R.mz + 1 >= R.nz) ? R.nz - 1 : R.mz;
    const float lr2 = (float)d.m_rc2;
    // the atom's place inside its own sector, for skipping whole sectors
    // beyond the list radius (only where the search range is a true offset
    // range, and with a margin far above float rounding)
    const double4_32a ri = d.r[i];
    const float ux = (float)(ri.x - sx * R.edge[0]), uy = (float)(ri.y - sy * R.edge[1]),
                uz = (float)(ri.z - sz * R.edge[2]);
    const float ex = (float)R.edge[0], ey = (float)R.edge[1], ez = (float)R.edge[2];
    const bool cx = 2 * R.mx + 1 < R.nx, cy = 2 * R.my + 1 < R.ny, cz = 2 * R.mz + 1 < R.nz;
    const float cut2 = lm2 * 1.001f;
    auto gap = [](bool on, int o, float u, float e) {
      if (!on || o == 0) return 0.0f;
      return o > 0 ? (float)o * e - u : u + (float)(-o - 1) * e;
    };
    int ce = 0, cc = 0, n1 = 0, c1 = 0, c2 = 0;
    // pass 0: exchange entries and the Morse-only entries certain to stay
    // inside the cutoff (counting those inside it at the build); pass 1: the
    // others, inside the cutoff at the build first, then beyond it
    for (int pass = 0; pass < 2; ++pass)
    for (int oz = loz; oz <= hiz; ++oz) {
      const float gz = gap(cz, oz, uz, ez);
      if (gz * gz > cut2) continue;
      int tz = (sz + oz + 2 * R.nz) % R.nz;
      for (int oy = loy; oy <= hiy; ++oy) {
        const float gy = gap(cy, oy, uy, ey);
        if (gz * gz + gy * gy > cut2) continue;
        int ty = (sy + oy + 2 * R.ny) % R.ny;
        for (int ox = lox; ox <= hix; ++ox) {
          const float gx = gap(cx, ox, ux, ex);
          if (gz * gz + gy * gy + gx * gx > cut2) continue;
          int tx = (sx + ox + 2 * R.nx) % R.nx;
          int q = sl_sector_rank(d, R, tx, ty, tz);
          int a = d.sec_start[q], b = d.sec_start[q + 1];
          for (int j = a; j < b; ++j) {
            if (j == i) continue;
            const float r2 = pair_pre(B, pi, load_pos(d, j)).r2;
            if (r2 < le2) {
              if (pass == 0) {
                if (ce < d.max_ex) d.exj[(size_t)ce * d.n + i] = j;
                ++ce;
              }
            } else if (r2 < lm2) {
              const int cls = r2 < lc2 ? 0 : (r2 < lr2 ? 1 : 2);
              // Morse-only entries go after a gap of max_ex rows for now
              int row = -1;
              if (pass == 0) {
                if (cls == 0) row = d.max_ex + cc++;
                else if (cls == 1) ++n1;
              } else if (cls == 1) {
                row = d.max_ex + cc + c1++;
              } else if (cls == 2) {
                row = d.max_ex + cc + n1 + c2++;
              }
              if (row >= 0 && row < d.max_m) d.mj[(size_t)row * d.n + i] = j;
            }
          }
        }
      }
    }
    const int cm = cc + c1 + c2;
    if (d.max_ex + cm > d.max_m || ce > d.max_ex) sl_set_error(d.ctrl, SL_ERR_NBR_OVERFLOW);
    const int ne = min(ce, d.max_ex);
    const int nmo = min(cm, d.max_m - d.max_ex);
    d.mn[i] = ne + nmo;
    d.mnc[i] = ne + min(cc, nmo);
    d.exn[i] = ne;
    // stable partition: same-sector neighbours first
    const int qi = d.secq[i];
    const int sa = d.sec_start[qi], sb = d.sec_start[qi + 1];
    int* col = d.exj + i;     // entry k at col[k * n]
    const size_t n = (size_t)d.n;
    int tmp[SL_MAX_EX_CAP];
    unsigned char tcol[SL_MAX_EX_CAP];
    int nin = 0, nout = 0;
    for (int k = 0; k < ne; ++k) {
      const int j = col[k * n];
      if (j >= sa && j < sb) col[(nin++) * n] = j;
      else tmp[nout++] = j;
    }
    // the other neighbours grouped by their sector's colour (stable); group c
    // starts at entry byte c of exc[i] (group 8 ends at exn[i])
    for (int k = 0; k < nout; ++k) tcol[k] = (unsigned char)(d.secq[tmp[k]] / d.s8);
    unsigned st[8];
    int w = nin;
    for (int c = 0; c < 8; ++c) {
      st[c] = (unsigned)w;
      for (int k = 0; k < nout; ++k)
        if (tcol[k] == c) col[(w++) * n] = tmp[k];
    }
    d.exc[i] = make_uint2(st[0] | st[1] << 8 | st[2] << 16 | st[3] << 24, st[4] | st[5] << 8 | st[6] << 16 | st[7] << 24);
    d.exin[i] = nin;
    // Morse list: the exchange list, then the Morse-only entries moved down
    int* mcol = d.mj + i;
    for (int k = 0; k < nmo; ++k) mcol[(ne + k) * n] = mcol[(d.max_ex + k) * n];
    for (int k = 0; k < ne; ++k) mcol[k * n] = col[k * n];
    atomicMax(&d.ctrl->max_m_seen, ce + cm);
    atomicMax(&d.ctrl->max_ex_seen, ce);
  }
}

// Dependency levels of the in-sector sweep (one thread per sector, after the
// lists): in sweep order a spin's rotation reads the already-turned spins of
// its same-sector list neighbours, so it can run at level 1 + the largest
// level of the neighbours before it (0 if none).  Spins of one level have no
// list edge between them and turn concurrently with the same result as the
// sequential order.  Forward order is ascending sorted index, backward
// descending.  Levels above 255 are an overflow (SL_ERR_NBR_OVERFLOW).
__global__ void k_rb_levels(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  const size_t n = (size_t)d.n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.nsec; q += gridDim.x * blockDim.x) {
    const int a = d.sec_start[q], b = d.sec_start[q + 1];
    for (int i = a; i < b; ++i) {
      int lf = 0;
      const int ni = d.exin[i];
      for (int k = 0; k < ni; ++k) {
        const int j = d.exj[(size_t)k * n + i];
        if (j < i) lf = max(lf, (d.lvl[j] & 0xFF) + 1);
      }
      if (lf > 255) { sl_set_error(d.ctrl, SL_ERR_NBR_OVERFLOW); lf = 255; }
      d.lvl[i] = (unsigned short)lf;
    }
    for (int i = b - 1; i >= a; --i) {
      int lb = 0;
      const int ni = d.exin[i];
      for (int k = 0; k < ni; ++k) {
        const int j = d.exj[(size_t)k * n + i];
        if (j > i) lb = max(lb, (d.lvl[j] >> 8) + 1);
      }
      if (lb > 255) { sl_set_error(d.ctrl, SL_ERR_NBR_OVERFLOW); lb = 255; }
      d.lvl[i] = (unsigned short)((d.lvl[i] & 0xFF) | (lb << 8));
    }
  }
}

__global__ void k_rb_end(SlDev d) {
  if (!d.ctrl->need_rebuild) return;
  d.ctrl->need_rebuild = 0;
  d.ctrl->rebuilds += 1;
}

__global__ void k_force_rebuild_flag(SlDev d) {
  d.ctrl->need_rebuild = 1;
  d.ctrl->maxdisp2_bits = 0ull;
}

inline int grid_for(int n) { return (n + SL_BLOCK - 1) / SL_BLOCK; }

}  // namespace

int sl_launch_force_rebuild_flag(const SlDev& d, cudaStream_t st) {
  k_force_rebuild_flag<<<1, 1, 0, st>>>(d);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

// The rebuild sequence; each kernel returns at once unless need_rebuild is set.
// The per-atom and per-sector kernels loop over a grid of at most rb_cap
// blocks: on the many steps without a rebuild they only launch and return.
int sl_launch_rebuild(const SlDev& d, cudaStream_t st) {
  const int cap = d.rb_cap > 0 ? d.rb_cap : 1 << 30;
  int gn = std::min(grid_for(d.n), cap), gs = std::min(grid_for(d.nsec), cap);
  int gz = gs < 1024 ? gs : 1024;
  k_rb_zero<<<gz, SL_BLOCK, 0, st>>>(d);
  k_rb_assign<<<gn, SL_BLOCK, 0, st>>>(d);
  k_rb_scan<<<1, 1024, 0, st>>>(d);
  k_rb_scatter<<<gn, SL_BLOCK, 0, st>>>(d);
  k_rb_sort<<<gs, SL_BLOCK, 0, st>>>(d);
  k_rb_gather<<<gn, SL_BLOCK, 0, st>>>(d);
  k_rb_copyback<<<gn, SL_BLOCK, 0, st>>>(d);
  sl_launch_split(d, st, 1);
  k_rb_nbr<<<gn, SL_BLOCK, 0, st>>>(d);
  k_rb_levels<<<gs, SL_BLOCK, 0, st>>>(d);
  k_rb_end<<<1, 1, 0, st>>>(d);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
