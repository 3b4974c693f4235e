// Cell binning and the two Verlet lists of the RelRes pair computation.
//
// Section 2.6 of the paper: the speedup of RelRes comes from keeping two
// neighbour lists with different cutoffs -- every atom lists its near
// neighbours within r_s+ (+ skin) for the FG part, and only hybrid sites list
// each other within r_c+ (+ skin) for the CG part.  Here both lists are full
// (each pair stored on both atoms, so the pair kernels write every force
// exactly once without atomics), column-major (entry k of slot s at k*n + s,
// so a warp's 32 index loads are one 128-byte transaction), and hold sorted
// slot indices: atoms are counting-sorted into cells visited in Morton order,
// which keeps the position gathers of the pair kernels local in L1/L2.
//
// Rebuild sequence: k_bin (cell of every atom, counts) -> k_scan (exclusive
// scan per grid) -> k_scatter (slot = start + atomic cursor) -> k_sort_cells
// (atom order inside each cell, so lists are deterministic) -> k_pack (sorted
// positions, ranks, reference positions for the displacement trigger) ->
// k_list (FG and CG lists).  Every kernel can be gated on the device rebuild
// flag, so the whole sequence can sit inside a CUDA graph step.
#include "common.cuh"

namespace relres {

struct GridArgs {
  int n0, n1, n2, ncell;
  int valid;  // 0: the grid is not used (no CG interaction); pointers are stand-ins
  const int* rank_of;
  int* start;
  int* count;
};

static GridArgs grid_args(const Grid& g) {
  return GridArgs{g.n[0], g.n[1], g.n[2], g.ncell, 1, g.d_rank_of, g.d_start, g.d_count};
}

// The binning kernels take plain scalar and pointer parameters only.  A
// version that passed its two grid descriptor structs by value into an inlined
// helper computed wrong cells (every atom in x-cell 0) or faulted on sm_103a,
// although a probe with the same signature read every field correctly; this
// form has no struct parameters at all.
__device__ __forceinline__ int linear_cell(int h0, int h1, int h2, int n0, int n1, int n2) {
  return (cell_of(h0, n0) * n1 + cell_of(h1, n1)) * n2 + cell_of(h2, n2);
}

// Cell (dense Morton rank) of every atom in each grid, and its arrival rank
// inside that cell (the value the count had before this atom was added).
__global__ void k_bin(int n, const unsigned* gate, const unsigned long long* __restrict__ xfx,
                      const int* __restrict__ type, int hyb_mask, int f0, int f1, int f2,
                      const int* __restrict__ frank, int* fcount, int with_cg, int c0, int c1, int c2,
                      const int* __restrict__ crank, int* ccount, int* __restrict__ cell_fg,
                      int* __restrict__ slot_fg, int* __restrict__ cell_cg, int* __restrict__ slot_cg,
                      unsigned* flags) {
  if (gate_closed(gate)) return;
  const int nf = f0 * f1 * f2, nc = c0 * c1 * c2;
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int h0 = hi32(xfx[3 * i]), h1 = hi32(xfx[3 * i + 1]), h2 = hi32(xfx[3 * i + 2]);
    // self-check: every index is tested before it is used (a failure is
    // reported through F_BADCELL and the access skipped)
    // (an atom with a bad index is still counted, in cell 0, so that the
    // later stages stay consistent and in bounds)
    const int lf = linear_cell(h0, h1, h2, f0, f1, f2);
    int cf = (lf >= 0 && lf < nf) ? frank[lf] : -1;
    if (cf < 0 || cf >= nf) {
      bad = true;
      cf = 0;
    }
    cell_fg[i] = cf;
    slot_fg[i] = atomicAdd(fcount + cf, 1);
    if (with_cg && ((hyb_mask >> type[i]) & 1)) {
      const int lc = linear_cell(h0, h1, h2, c0, c1, c2);
      int cc = (lc >= 0 && lc < nc) ? crank[lc] : -1;
      if (cc < 0 || cc >= nc) {
        bad = true;
        cc = 0;
      }
      cell_cg[i] = cc;
      slot_cg[i] = atomicAdd(ccount + cc, 1);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, F_BADCELL);
}

// One block per grid: exclusive scan of counts into start[0..ncell], counts
// reset to zero (they become the scatter cursors).
__global__ void k_scan(const unsigned* gate, int valid0, int ncell0, int* start0, int* count0, int valid1,
                       int ncell1, int* start1, int* count1, DevState* st) {
  if (gate_closed(gate)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // list statistics of this build
    st->max_fg = 0;
    st->max_cg = 0;
    st->tot_fg = 0;
    st->tot_cg = 0;
  }
  const int valid = blockIdx.x == 0 ? valid0 : valid1;
  const int ncell = blockIdx.x == 0 ? ncell0 : ncell1;
  int* const start = blockIdx.x == 0 ? start0 : start1;
  int* const count = blockIdx.x == 0 ? count0 : count1;
  if (!valid) return;
  __shared__ int sh[1024 / 32];
  const int nt = blockDim.x;
  const int per = (ncell + nt - 1) / nt;
  const int b = threadIdx.x * per, e = min(ncell, b + per);
  int local = 0;
  for (int c = b; c < e; ++c) local += count[c];
  // block exclusive scan of `local`
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = lane < (nt >> 5) ? sh[lane] : 0;
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, iv, o);
      if (lane >= o) iv += t;
    }
    if (lane < (nt >> 5)) sh[lane] = iv - v;
  }
  __syncthreads();
  int run = sh[wid] + incl - local;
  for (int c = b; c < e; ++c) {
    const int k = count[c];
    start[c] = run;
    count[c] = 0;
    run += k;
  }
  if (threadIdx.x == nt - 1) start[ncell] = run;
}

__global__ void k_scatter(int n, const unsigned* gate, const int* __restrict__ type, int hyb_mask,
                          const int* __restrict__ fstart, int with_cg, const int* __restrict__ cstart,
                          const int* __restrict__ cell_fg, const int* __restrict__ slot_fg,
                          const int* __restrict__ cell_cg, const int* __restrict__ slot_cg,
                          int* __restrict__ perm_fg, int* __restrict__ perm_cg) {
  if (gate_closed(gate)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    perm_fg[fstart[cell_fg[i]] + slot_fg[i]] = i;
    if (with_cg && ((hyb_mask >> type[i]) & 1)) perm_cg[cstart[cell_cg[i]] + slot_cg[i]] = i;
  }
}

// One thread per cell: insertion-sort the cell's atoms by index (the scatter
// order is arbitrary), reset the cursor.
__global__ void k_sort_cells(const unsigned* gate, int fn, const int* fstart, int* fcount, int cn,
                             const int* cstart, int* ccount, int* __restrict__ perm_fg,
                             int* __restrict__ perm_cg) {
  if (gate_closed(gate)) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < fn + cn; t += gridDim.x * blockDim.x) {
    const bool fg = t < fn;
    const int c = fg ? t : t - fn;
    const int* const start = fg ? fstart : cstart;
    int* const count = fg ? fcount : ccount;
    int* const perm = fg ? perm_fg : perm_cg;
    const int lo = start[c], hi = start[c + 1];
    for (int k = lo + 1; k < hi; ++k) {
      const int v = perm[k];
      int m = k - 1;
      while (m >= lo && perm[m] > v) {
        perm[m + 1] = perm[m];
        --m;
      }
      perm[m + 1] = v;
    }
    count[c] = 0;
  }
}

__global__ void k_pack(int n, int n_h, const unsigned* gate, const unsigned long long* __restrict__ xfx,
                       const int* __restrict__ type, const int* __restrict__ perm_fg,
                       const int* __restrict__ perm_cg, int* __restrict__ rank_fg,
                       int* __restrict__ rank_cg, int4* __restrict__ pos_fg,
                       int4* __restrict__ pos_cg, Pos64* __restrict__ pos_fg64,
                       Pos64* __restrict__ pos_cg64, int fp64, int4* __restrict__ ref) {
  if (gate_closed(gate)) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int i = perm_fg[s];
    const unsigned long long x = xfx[3 * i], y = xfx[3 * i + 1], z = xfx[3 * i + 2];
    const int t = type[i];
    rank_fg[i] = s;
    const int4 h = make_int4(hi32(x), hi32(y), hi32(z), t);
    pos_fg[s] = h;
    ref[i] = h;
    if (fp64) pos_fg64[s] = Pos64{(long long)x, (long long)y, (long long)z, t};
    if (s < n_h) {
      const int j = perm_cg[s];
      const unsigned long long xj = xfx[3 * j], yj = xfx[3 * j + 1], zj = xfx[3 * j + 2];
      rank_cg[j] = s;
      pos_cg[s] = make_int4(hi32(xj), hi32(yj), hi32(zj), type[j]);
      if (fp64) pos_cg64[s] = Pos64{(long long)xj, (long long)yj, (long long)zj, type[j]};
    }
  }
}

struct ListArgs {
  int nslots;
  const int4* pos;
  const int* perm;
  GridArgs g;
  float sx, sy, sz;
  float rl2;
  const int* excl_off;
  const int* excl_idx;
  int cap;
  int* nbr;
  int* cnt;
  int* max_out;
  unsigned long long* total_out;
  unsigned* flags;
  unsigned overflow_bit;
};

__device__ __forceinline__ int axis_cells(int c, int n, int (&out)[3]) {
  if (n >= 3) {
    out[0] = c == 0 ? n - 1 : c - 1;
    out[1] = c;
    out[2] = c == n - 1 ? 0 : c + 1;
    return 3;
  }
  for (int k = 0; k < n; ++k) out[k] = k;  // 1 or 2 cells: visit each once
  return n;
}

__global__ void __launch_bounds__(kThreads) k_list(const unsigned* gate, ListArgs a) {
  if (gate_closed(gate)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nslots) return;
  const int4 p = a.pos[s];
  const int i = a.perm[s];
  const int e0 = a.excl_off ? a.excl_off[i] : 0;
  const int e1 = a.excl_off ? a.excl_off[i + 1] : 0;
  int cx[3], cy[3], cz[3];
  const int nx = axis_cells(cell_of(p.x, a.g.n0), a.g.n0, cx);
  const int ny = axis_cells(cell_of(p.y, a.g.n1), a.g.n1, cy);
  const int nz = axis_cells(cell_of(p.z, a.g.n2), a.g.n2, cz);
  int count = 0;
  // entries are stored in chunks of four (one 16-byte store per chunk):
  // entry k of slot s at int (((k >> 2) * nslots + s) << 2) + (k & 3)
  int4* const out4 = reinterpret_cast<int4*>(a.nbr) + s;
  int4 buf = make_int4(s, s, s, s);
  for (int ix = 0; ix < nx; ++ix)
    for (int iy = 0; iy < ny; ++iy)
      for (int iz = 0; iz < nz; ++iz) {
        const int c = a.g.rank_of[(cx[ix] * a.g.n1 + cy[iy]) * a.g.n2 + cz[iz]];
        const int tb = a.g.start[c], te = a.g.start[c + 1];
        for (int t = tb; t < te; ++t) {
          if (t == s) continue;
          const int4 q = a.pos[t];
          const float dx = dfix32(p.x, q.x, a.sx);
          const float dy = dfix32(p.y, q.y, a.sy);
          const float dz = dfix32(p.z, q.z, a.sz);
          if (dx * dx + dy * dy + dz * dz >= a.rl2) continue;
          if (e1 > e0) {
            const int j = a.perm[t];
            bool ex = false;
            for (int e = e0; e < e1; ++e) ex |= (a.excl_idx[e] == j);
            if (ex) continue;
          }
          if (count < a.cap) {
            const int q = count & 3;
            buf.x = q == 0 ? t : buf.x;
            buf.y = q == 1 ? t : buf.y;
            buf.z = q == 2 ? t : buf.z;
            buf.w = q == 3 ? t : buf.w;
            if (q == 3) out4[size_t(count >> 2) * a.nslots] = buf;
          }
          ++count;
        }
      }
  // the last partial chunk (its padding lanes hold earlier indices, never read as partners)
  const int kept = min(count, a.cap);
  if (kept & 3) out4[size_t(kept >> 2) * a.nslots] = buf;
  a.cnt[s] = kept;
  atomicMax(a.max_out, count);
  atomicAdd(a.total_out, (unsigned long long)count);
  if (count > a.cap) atomicOr(a.flags, a.overflow_bit);
}

static int blocks_for(int n) {
  const int b = (n + kThreads - 1) / kThreads;
  return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

cudaError_t launch_rebuild(relres_ctx* c, const unsigned* gate) {
  if (gate == nullptr) gate = c->d_open;
  const GridArgs gf = grid_args(c->gfg);
  GridArgs gc = grid_args(c->gcg);
  if (!c->has_cg || c->n_h == 0) {
    gc = gf;  // stand-in pointers, never used
    gc.valid = 0;
  }
  Pos64* p64f = c->fp64 ? c->d_pos_fg64 : static_cast<Pos64*>(c->d_dummy);
  Pos64* p64c = c->fp64 ? c->d_pos_cg64 : static_cast<Pos64*>(c->d_dummy);
  const int nb = blocks_for(c->n);
  k_bin<<<nb, kThreads, 0, c->stream>>>(c->n, gate, c->d_xfx, c->d_type, c->hyb_mask, gf.n0, gf.n1,
                                        gf.n2, gf.rank_of, gf.count, gc.valid, gc.n0, gc.n1, gc.n2,
                                        gc.rank_of, gc.count, c->d_cell_fg, c->d_slot_fg, c->d_cell_cg,
                                        c->d_slot_cg, &c->d_state->flags);
  RELRES_LAUNCHED(c);
  k_scan<<<2, 1024, 0, c->stream>>>(gate, 1, gf.ncell, gf.start, gf.count, gc.valid, gc.ncell, gc.start,
                                    gc.count, c->d_state);
  RELRES_LAUNCHED(c);
  k_scatter<<<nb, kThreads, 0, c->stream>>>(c->n, gate, c->d_type, c->hyb_mask, gf.start, gc.valid, gc.start,
                                            c->d_cell_fg, c->d_slot_fg, c->d_cell_cg, c->d_slot_cg,
                                            c->d_perm_fg, c->d_perm_cg);
  RELRES_LAUNCHED(c);
  const int ncells = gf.ncell + (gc.valid ? gc.ncell : 0);
  k_sort_cells<<<blocks_for(ncells), kThreads, 0, c->stream>>>(gate, gf.ncell, gf.start, gf.count,
                                                               gc.valid ? gc.ncell : 0, gc.start, gc.count,
                                                               c->d_perm_fg, c->d_perm_cg);
  RELRES_LAUNCHED(c);
  k_pack<<<nb, kThreads, 0, c->stream>>>(c->n, gc.valid ? c->n_h : 0, gate, c->d_xfx, c->d_type,
                                         c->d_perm_fg, c->d_perm_cg, c->d_rank_fg, c->d_rank_cg,
                                         c->d_pos_fg, c->d_pos_cg, p64f, p64c, c->fp64 ? 1 : 0, c->d_ref);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_lists(relres_ctx* c, const unsigned* gate) {
  if (gate == nullptr) gate = c->d_open;
  const float s0 = float(c->box[0] / 4294967296.0), s1 = float(c->box[1] / 4294967296.0),
              s2 = float(c->box[2] / 4294967296.0);
  DevState* st = c->d_state;
  {
    const double rl = c->rlist_fg_cut + c->prm.skin;
    ListArgs a{c->n, c->d_pos_fg, c->d_perm_fg, grid_args(c->gfg), s0, s1, s2, float(rl * rl),
               c->d_excl_off, c->d_excl_idx, c->cap_fg, c->d_nbr_fg, c->d_cnt_fg, &st->max_fg,
               &st->tot_fg, &st->flags, F_OVERFLOW_FG};
    k_list<<<(c->n + kThreads - 1) / kThreads, kThreads, 0, c->stream>>>(gate, a);
    RELRES_LAUNCHED(c);
  }
  if (c->has_cg && c->n_h > 0) {
    const double rl = c->rlist_cg_cut + c->skin_cg;
    ListArgs a{c->n_h, c->d_pos_cg, c->d_perm_cg, grid_args(c->gcg), s0, s1, s2, float(rl * rl),
               c->d_excl_off, c->d_excl_idx, c->cap_cg, c->d_nbr_cg, c->d_cnt_cg, &st->max_cg,
               &st->tot_cg, &st->flags, F_OVERFLOW_CG};
    k_list<<<(c->n_h + kThreads - 1) / kThreads, kThreads, 0, c->stream>>>(gate, a);
    RELRES_LAUNCHED(c);
  }
  return cudaGetLastError();
}

}  // namespace relres
