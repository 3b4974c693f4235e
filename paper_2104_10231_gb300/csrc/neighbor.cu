// Cell binning and the two Verlet lists of the RelRes pair computation.
//
// Section 2.6 of the paper: the speedup of RelRes comes from keeping two
// neighbour lists with different cutoffs -- every atom lists its near
// neighbours within r_s+ (+ skin) for the FG part, and only hybrid sites list
// each other within r_c+ (+ skin) for the CG part.  Here both lists are full
// (each pair stored on both atoms, so the pair kernel writes every force
// exactly once without atomics), stored in chunks of four entries per slot
// (entry k of slot s at int (((k >> 2) * nslots + s) << 2) + (k & 3), so a
// warp reads 512 contiguous bytes per chunk), and hold sorted slot indices:
// atoms are counting-sorted into cells visited in Morton order, which keeps
// the position gathers of the pair kernel local in L1/L2.
//
// Rebuild sequence: k_bin (cell of every atom, counts) -> k_scan (exclusive
// scan per grid) -> k_scatter (slot = start + arrival rank) -> k_sort_cells
// (atom order inside each cell, so lists are deterministic) -> k_pack (sorted
// positions, ranks, reference positions for the displacement trigger) ->
// k_list (FG and CG lists in one launch).  Every kernel can be gated on the
// device rebuild flag, so the whole sequence can sit inside a CUDA graph step.
// The pair kernels walk pruned copies of the lists (k_prune below, or the pair
// kernel's own pruning walk).
#include "common.cuh"

namespace relres {

struct GridArgs {
  int n0, n1, n2, ncell;
  int valid;  // 0: the grid is not used (no CG interaction); pointers are stand-ins
  const int* rank_of;
  int* start;
  int* count;
  int nf0, nf1, nf2, xsplit, ncell_full, ntile;
  int* tile;
};

static GridArgs grid_args(const Grid& g) {
  return GridArgs{g.n[0], g.n[1], g.n[2], g.ncell, 1, g.d_rank_of, g.d_start, g.d_count,
                  g.nf[0], g.nf[1], g.nf[2], g.xsplit, g.ncell_full, g.ntile, g.d_tile};
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
// (block bid of nblk; the single-system kernel passes blockIdx.x, gridDim.x)
__device__ __forceinline__ void bin_body(int bid, int nblk, int n, const unsigned* gate,
                                        const unsigned long long* __restrict__ xfx, const int* __restrict__ type,
                                        int hyb_mask, int f0, int f1, int f2, const int* __restrict__ frank,
                                        int* fcount, int with_cg, int c0, int c1, int c2,
                                        const int* __restrict__ crank, int* ccount, int* __restrict__ cell_fg,
                                        int* __restrict__ slot_fg, int* __restrict__ cell_cg,
                                        int* __restrict__ slot_cg, unsigned* flags) {
  if (gate_closed(gate)) return;
  const int nf = f0 * f1 * f2, nc = c0 * c1 * c2;
  bool bad = false;
  for (int i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
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

__global__ void k_bin(int n, const unsigned* gate, const unsigned long long* __restrict__ xfx,
                      const int* __restrict__ type, int hyb_mask, int f0, int f1, int f2,
                      const int* __restrict__ frank, int* fcount, int with_cg, int c0, int c1, int c2,
                      const int* __restrict__ crank, int* ccount, int* __restrict__ cell_fg,
                      int* __restrict__ slot_fg, int* __restrict__ cell_cg, int* __restrict__ slot_cg,
                      unsigned* flags) {
  bin_body(blockIdx.x, gridDim.x, n, gate, xfx, type, hyb_mask, f0, f1, f2, frank, fcount, with_cg, c0, c1, c2,
           crank, ccount, cell_fg, slot_fg, cell_cg, slot_cg, flags);
}

// Exclusive scan of the cell counts into start[0..ncell] in two passes over
// tiles of kScanTile cells: scan_tile_body scans one tile locally (4 cells per
// thread of 1024, warp shuffles, then the warp totals), writes the tile total
// and resets the counts to zero for the next build; scan_add_body adds the sum
// of the tile totals before its tile.  Tile t of a build: the tiles of the FG
// grid, then those of the CG grid.
struct ScanGrid {
  int valid, ncell, ntile;
  int* start;
  int* count;
  int* tile;
};

__device__ __forceinline__ void pick_scan(const ScanGrid& g0, const ScanGrid& g1, int t, ScanGrid* g, int* tile) {
  if (t < g0.ntile) {
    *g = g0;
    *tile = t;
  } else {
    *g = g1;
    *tile = t - g0.ntile;
  }
}

__device__ __forceinline__ void scan_tile_body(int t, const unsigned* gate, const ScanGrid& g0, const ScanGrid& g1,
                                              DevState* st) {
  if (gate_closed(gate)) return;
  if (t == 0 && threadIdx.x == 0) {  // list statistics of this build
    st->max_fg = 0;
    st->max_cg = 0;
    st->tot_fg = 0;
    st->tot_cg = 0;
  }
  ScanGrid g;
  int tile;
  pick_scan(g0, g1, t, &g, &tile);
  __shared__ int sh[kScanTile / 4 / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int c0 = tile * kScanTile + 4 * threadIdx.x;
  int v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = c0 + q < g.ncell ? g.count[c0 + q] : 0;
  const int tsum = v[0] + v[1] + v[2] + v[3];
  int incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sh[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < nw) sh[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  int run = (wid > 0 ? sh[wid - 1] : 0) + incl - tsum;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (c0 + q < g.ncell) {
      g.start[c0 + q] = run;
      g.count[c0 + q] = 0;
      run += v[q];
    }
  if (threadIdx.x == 0) g.tile[tile] = sh[nw - 1];
  __syncthreads();  // sh is reused by a batched kernel's next work item
}

__device__ __forceinline__ void scan_add_body(int t, const unsigned* gate, const ScanGrid& g0, const ScanGrid& g1) {
  if (gate_closed(gate)) return;
  ScanGrid g;
  int tile;
  pick_scan(g0, g1, t, &g, &tile);
  __shared__ int sh[kScanTile / 4 / 32];
  int part = 0;
  for (int u = threadIdx.x; u < tile; u += blockDim.x) part += g.tile[u];
  part = warp_sum(part);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[wid] = part;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < nw; ++w) off += sh[w];
  const int c0 = tile * kScanTile + 4 * threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (c0 + q < g.ncell) g.start[c0 + q] += off;
  if (tile == g.ntile - 1 && threadIdx.x == 0) g.start[g.ncell] = off + g.tile[tile];
  __syncthreads();  // sh is reused by a batched kernel's next work item
}

__global__ void __launch_bounds__(kScanTile / 4) k_scan_tiles(const unsigned* gate, ScanGrid g0, ScanGrid g1,
                                                               DevState* st) {
  scan_tile_body(blockIdx.x, gate, g0, g1, st);
}

__global__ void __launch_bounds__(kScanTile / 4) k_scan_add(const unsigned* gate, ScanGrid g0, ScanGrid g1) {
  scan_add_body(blockIdx.x, gate, g0, g1);
}

__host__ __device__ __forceinline__ ScanGrid scan_grid(const GridArgs& g) {
  return ScanGrid{g.valid, g.ncell, g.valid ? g.ntile : 0, g.start, g.count, g.tile};
}

__device__ __forceinline__ void scatter_body(int bid, int nblk, int n, const unsigned* gate,
                                            const int* __restrict__ type, int hyb_mask,
                                            const int* __restrict__ fstart, int with_cg,
                                            const int* __restrict__ cstart, const int* __restrict__ cell_fg,
                                            const int* __restrict__ slot_fg, const int* __restrict__ cell_cg,
                                            const int* __restrict__ slot_cg, int* __restrict__ perm_fg,
                                            int* __restrict__ perm_cg) {
  if (gate_closed(gate)) return;
  for (int i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    perm_fg[fstart[cell_fg[i]] + slot_fg[i]] = i;
    if (with_cg && ((hyb_mask >> type[i]) & 1)) perm_cg[cstart[cell_cg[i]] + slot_cg[i]] = i;
  }
}

__global__ void k_scatter(int n, const unsigned* gate, const int* __restrict__ type, int hyb_mask,
                          const int* __restrict__ fstart, int with_cg, const int* __restrict__ cstart,
                          const int* __restrict__ cell_fg, const int* __restrict__ slot_fg,
                          const int* __restrict__ cell_cg, const int* __restrict__ slot_cg,
                          int* __restrict__ perm_fg, int* __restrict__ perm_cg) {
  scatter_body(blockIdx.x, gridDim.x, n, gate, type, hyb_mask, fstart, with_cg, cstart, cell_fg, slot_fg, cell_cg,
               slot_cg, perm_fg, perm_cg);
}

// One thread per cell: the cell's atoms put in index order (the scatter order
// is arbitrary) by an insertion sort in place; cells hold ~5 atoms.
__device__ __forceinline__ void sort_body(int bid, int nblk, const unsigned* gate, int fn, const int* fstart, int cn,
                                         const int* cstart, int* __restrict__ perm_fg, int* __restrict__ perm_cg) {
  if (gate_closed(gate)) return;
  for (int t = bid * blockDim.x + threadIdx.x; t < fn + cn; t += nblk * blockDim.x) {
    const bool fg = t < fn;
    const int c = fg ? t : t - fn;
    const int* const start = fg ? fstart : cstart;
    int* const perm = fg ? perm_fg : perm_cg;
    const int lo = start[c], hi = start[c + 1];
    for (int k = lo + 1; k < hi; ++k) {
      const int v = perm[k];
      int q = k - 1;
      int u = perm[q];
      while (u > v) {
        perm[q + 1] = u;
        if (--q < lo) break;
        u = perm[q];
      }
      perm[q + 1] = v;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_sort_cells(const unsigned* gate, int fn, const int* fstart, int cn,
                                                         const int* cstart, int* __restrict__ perm_fg,
                                                         int* __restrict__ perm_cg) {
  sort_body(blockIdx.x, gridDim.x, gate, fn, fstart, cn, cstart, perm_fg, perm_cg);
}

__device__ __forceinline__ void pack_body(int bid, int nblk, int n, int n_h, const unsigned* gate,
                                         const unsigned long long* __restrict__ xfx, const int* __restrict__ type,
                                         const int* __restrict__ perm_fg, const int* __restrict__ perm_cg,
                                         int* __restrict__ rank_fg, int* __restrict__ rank_cg,
                                         int4* __restrict__ pos_fg, int4* __restrict__ pos_cg,
                                         Pos64* __restrict__ pos_fg64, Pos64* __restrict__ pos_cg64, int fp64,
                                         int4* __restrict__ ref) {
  if (gate_closed(gate)) return;
  for (int s = bid * blockDim.x + threadIdx.x; s < n; s += nblk * blockDim.x) {
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

__global__ void k_pack(int n, int n_h, const unsigned* gate, const unsigned long long* __restrict__ xfx,
                       const int* __restrict__ type, const int* __restrict__ perm_fg,
                       const int* __restrict__ perm_cg, int* __restrict__ rank_fg,
                       int* __restrict__ rank_cg, int4* __restrict__ pos_fg,
                       int4* __restrict__ pos_cg, Pos64* __restrict__ pos_fg64,
                       Pos64* __restrict__ pos_cg64, int fp64, int4* __restrict__ ref) {
  pack_body(blockIdx.x, gridDim.x, n, n_h, gate, xfx, type, perm_fg, perm_cg, rank_fg, rank_cg, pos_fg, pos_cg,
            pos_fg64, pos_cg64, fp64, ref);
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
  int excl_window;  // every excluded pair (i, j) has |i - j| <= excl_window (atom ids)
  int cap;
  int* nbr;
  int* cnt;
  int* max_out;
  unsigned long long* total_out;
  unsigned* flags;
  unsigned overflow_bit;
  // per-atom exclusion masks (bit j - i + kExclMaskHalf), or NULL: then the
  // exclusion lists are searched (excl_window above kExclMaskHalf)
  const unsigned* excl_mask;
};

constexpr int kListThreads = 128;  // 4 warps per cell

__device__ __forceinline__ float wrap1(float d, float l, float il) { return d - l * rintf(d * il); }

// One cell atom (slot s, atom id ai, relative position p) against the staged
// candidates beg .. end - 1 of the window: 32 candidates per iteration,
// accepted ones appended at k in window order.  A lane past `end` reads either
// a staged candidate of an x-slab beyond the atom's list radius (farther than
// the list radius by construction of the slab run) or the NaN padding after
// the window, so the distance test alone rejects it.  Exclusions: with MASK,
// bit aj - ai + kExclMaskHalf of the atom's mask (its own bit included); else
// a candidate whose atom id lies within the exclusion window of ai (this
// includes ai itself) is checked against ai's exclusion list, and all others
// cannot be excluded.  Returns the new count.
template <bool WRAP, bool MASK>
__device__ __forceinline__ int scan_range(const float4* s_pos, const int* s_atom, int beg, int end, int ai,
                                          float px, float py, float pz, float rl2, float lx, float ly,
                                          float lz, unsigned emask, const int (&ex)[8], int e0, int e1,
                                          const int* excl_idx, int win, int* nbr_s, unsigned stride, int cap,
                                          int k) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  for (int j0 = beg; j0 < end; j0 += 32) {
    const int j = j0 + lane;
    const float4 q = s_pos[j];
    float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    if (WRAP) {
      dx = wrap1(dx, lx, 1.f / lx);
      dy = wrap1(dy, ly, 1.f / ly);
      dz = wrap1(dz, lz, 1.f / lz);
    }
    bool acc = dx * dx + dy * dy + dz * dz < rl2;
    const int aj = s_atom[j];
    if (MASK) {
      const unsigned d = unsigned(aj - ai + kExclMaskHalf);
      acc = acc && !(d < unsigned(2 * kExclMaskHalf + 1) && ((emask >> d) & 1u));
    } else if (acc && unsigned(aj - ai + win) <= unsigned(2 * win)) {
      // the first eight excluded partners are in registers (-1 where unused)
      acc = aj != ai;
#pragma unroll
      for (int e = 0; e < 8; ++e) acc = acc && ex[e] != aj;
      for (int e = e0 + 8; e < e1; ++e) acc = acc && excl_idx[e] != aj;
    }
    const unsigned b = __ballot_sync(0xffffffffu, acc);
    const int kk = k + __popc(b & below);
    // entry kk of this slot: int ((kk >> 2) * nslots + s) * 4 + (kk & 3)
    if (acc && kk < cap) nbr_s[unsigned(kk >> 2) * stride + unsigned(kk & 3)] = __float_as_int(q.w);
    k += __popc(b);
  }
  return k;
}

constexpr int kListWindow = 1024;  // candidates staged in shared memory at a time (a multiple of 32)
constexpr int kListGroup = 64;     // cell atoms handled per pass

constexpr int kStageMax = 3 * kXSplit * 9;  // staged cells: 3 x kXSplit x-slabs by 3 by 3 cells

// One block per full cell (CG-grid cells first, then FG-grid cells).  The
// block stages the atoms of the 27 full cells around its cell in shared
// memory, x-slab after x-slab (on a split grid each full cell is kXSplit
// slabs along x), as FP32 coordinates relative to the cell's first atom (from
// the exact wrapped 32-bit differences; the list radius carries the skin, so
// FP32 rounding near the list radius cannot lose a pair inside the interaction
// range).  Each warp then takes one atom of the cell at a time and tests 32
// staged candidates per iteration: on a split grid only the run of x-slabs
// within the list radius of the atom (a contiguous range of the staged
// candidates, about 3/4 of them), otherwise all of them.  Accepted candidates
// are appended in staging order (ballot + prefix count), so the list is
// deterministic.
__device__ __forceinline__ void list_cell(const ListArgs& fg, const ListArgs& cg, int ncell_cg, int cb) {
  // x, y, z relative, w = slot index bits; atom ids; 32 NaN entries after the window
  __shared__ float4 s_pos[kListWindow + 32];
  __shared__ int s_atom[kListWindow + 32];
  __shared__ int s_cstart[kStageMax], s_coff[kStageMax + 1];
  __shared__ int s_k[kListGroup];
  // the group's atoms, read once per group: relative position (w = atom id
  // bits), exclusion mask, run [beg, end) of staged candidates
  __shared__ float4 s_gp[kListGroup];
  __shared__ unsigned s_gm[kListGroup];
  __shared__ int2 s_gr[kListGroup];
  __shared__ int s_max;
  __shared__ unsigned long long s_tot;
  const bool is_cg = cb < ncell_cg;
  // the list of this block, field by field (parameters are only read directly)
  struct {
    int nslots;
    const int4* pos;
    const int* perm;
    int excl_window;
    int n0, n1, n2, nf0, nf1, nf2, xsplit;
    const int* rank_of;
    const int* start;
    float sx, sy, sz, rl2;
    const int* excl_off;
    const int* excl_idx;
    int cap;
    int* nbr;
    int* cnt;
    int* max_out;
    unsigned long long* total_out;
    unsigned* flags;
    unsigned overflow_bit;
    const unsigned* excl_mask;
  } a;
#define RELRES_PICK(f) a.f = is_cg ? cg.f : fg.f
  RELRES_PICK(nslots);
  RELRES_PICK(pos);
  RELRES_PICK(perm);
  RELRES_PICK(excl_window);
  RELRES_PICK(sx);
  RELRES_PICK(sy);
  RELRES_PICK(sz);
  RELRES_PICK(rl2);
  RELRES_PICK(excl_off);
  RELRES_PICK(excl_idx);
  RELRES_PICK(cap);
  RELRES_PICK(nbr);
  RELRES_PICK(cnt);
  RELRES_PICK(max_out);
  RELRES_PICK(total_out);
  RELRES_PICK(flags);
  RELRES_PICK(overflow_bit);
  RELRES_PICK(excl_mask);
#undef RELRES_PICK
#define RELRES_PICKG(f) a.f = is_cg ? cg.g.f : fg.g.f
  RELRES_PICKG(n0);
  RELRES_PICKG(n1);
  RELRES_PICKG(n2);
  RELRES_PICKG(nf0);
  RELRES_PICKG(nf1);
  RELRES_PICKG(nf2);
  RELRES_PICKG(xsplit);
  RELRES_PICKG(rank_of);
  RELRES_PICKG(start);
#undef RELRES_PICKG
  const int S = a.xsplit;
  const int cf = is_cg ? cb : cb - ncell_cg;  // dense rank of the full cell
  const int i0 = a.start[cf * S];
  const int ni = a.start[(cf + 1) * S] - i0;
  if (ni == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int4 ref = a.pos[i0];
  // staged cells, x-major: per axis the full cells F-1, F, F+1 (x: as S slabs
  // each), or every cell of an axis with fewer than three
  const int fx = cell_of(ref.x, a.n0) / S, fy = cell_of(ref.y, a.n1), fz = cell_of(ref.z, a.n2);
  const int d0 = a.nf0 >= 3 ? 3 * S : a.n0, d1 = a.nf1 >= 3 ? 3 : a.n1, d2 = a.nf2 >= 3 ? 3 : a.n2;
  const int b0 = a.nf0 >= 3 ? S * (fx - 1) + a.n0 : 0, b1 = a.nf1 >= 3 ? fy - 1 + a.n1 : 0,
            b2 = a.nf2 >= 3 ? fz - 1 + a.n2 : 0;
  const int ms = d0 * d1 * d2;
  for (int t = threadIdx.x; t < ms; t += blockDim.x) {
    const int i = t / (d1 * d2), j = (t / d2) % d1, k = t % d2;
    const int gx = (b0 + i) % a.n0, gy = (b1 + j) % a.n1, gz = (b2 + k) % a.n2;
    const int cc = a.rank_of[(gx * a.n1 + gy) * a.n2 + gz];
    const int b = a.start[cc];
    s_cstart[t] = b;
    s_coff[t] = a.start[cc + 1] - b;  // count, scanned below
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the staged counts, up to 4 cells per lane
    const int per = (ms + 31) / 32;
    const int lo = min(ms, lane * per), hi = min(ms, lo + per);
    int sum = 0;
    for (int t = lo; t < hi; ++t) sum += s_coff[t];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    int run = incl - sum;
    for (int t = lo; t < hi; ++t) {
      const int cnt = s_coff[t];
      s_coff[t] = run;
      run += cnt;
    }
    if (lane == 31) s_coff[ms] = incl;
    if (lane == 0) {
      s_max = 0;
      s_tot = 0ull;
    }
  }
  __syncthreads();
  const int total = s_coff[ms];
  // With 4 or more full cells per axis every staged offset from the reference
  // atom and every candidate offset is below L/2, so plain differences of the
  // relative coordinates are minimum images; smaller grids wrap explicitly.
  const bool wrap = a.nf0 < 4 || a.nf1 < 4 || a.nf2 < 4;
  const bool slabs = S > 1 && !wrap;  // each atom tests its run of x-slabs only
  const float lx = a.sx * 4294967296.f, ly = a.sy * 4294967296.f, lz = a.sz * 4294967296.f;
  // list radius (+ a margin above the rounding of the positions) in x-slab widths
  const float reach = (sqrtf(a.rl2) + 1e-3f) * float(a.n0) / lx;
  const int slab_cells = d1 * d2;
  int blk_max = 0;
  unsigned long long blk_tot = 0ull;
  for (int g0 = 0; g0 < ni; g0 += kListGroup) {
    const int ng = min(kListGroup, ni - g0);
    for (int k = threadIdx.x; k < ng; k += blockDim.x) {
      s_k[k] = 0;
      const int s = i0 + g0 + k;
      const int4 p = a.pos[s];
      const int ai = a.perm[s];
      s_gp[k] = make_float4(dfix32(p.x, ref.x, a.sx), dfix32(p.y, ref.y, a.sy), dfix32(p.z, ref.z, a.sz),
                            __int_as_float(ai));
      s_gm[k] = a.excl_mask != nullptr ? a.excl_mask[ai] : 0u;
      int beg = 0, end = total;
      if (slabs) {
        // the atom's x in slab widths from the first staged slab: its own
        // slab (S .. 2S - 1) plus its place in it
        const int cx = cell_of(p.x, a.n0);
        const float ux = float(unsigned(p.x) * unsigned(a.n0)) * 2.3283064365386963e-10f;
        const float xs = float(cx - S * fx + S) + ux;
        const int lo = max(0, int(floorf(xs - reach))), hi = min(d0 - 1, int(floorf(xs + reach)));
        beg = s_coff[lo * slab_cells];
        end = s_coff[(hi + 1) * slab_cells];
      }
      s_gr[k] = make_int2(beg, end);
    }
    for (int w0 = 0; w0 < total; w0 += kListWindow) {
      const int wn = min(kListWindow, total - w0);
      __syncthreads();
      for (int k = threadIdx.x; k < wn; k += blockDim.x) {
        const int gidx = w0 + k;
        int m = 0;  // staged cell holding candidate gidx: the last one starting at or before it
#pragma unroll
        for (int step = 64; step > 0; step >>= 1)
          if (m + step < ms && s_coff[m + step] <= gidx) m += step;
        const int t = s_cstart[m] + (gidx - s_coff[m]);
        const int4 q = a.pos[t];
        s_pos[k] = make_float4(dfix32(q.x, ref.x, a.sx), dfix32(q.y, ref.y, a.sy), dfix32(q.z, ref.z, a.sz),
                               __int_as_float(t));
        s_atom[k] = a.perm[t];
      }
      if (threadIdx.x < 32) {  // padding read by the lanes past the end of a run
        const float nan = __int_as_float(0x7fc00000);
        s_pos[wn + threadIdx.x] = make_float4(nan, nan, nan, nan);
        s_atom[wn + threadIdx.x] = -1;
      }
      __syncthreads();
      for (int il = warp; il < ng; il += blockDim.x >> 5) {
        const int s = i0 + g0 + il;
        const float4 gp = s_gp[il];
        const float px = gp.x, py = gp.y, pz = gp.z;
        const int ai = __float_as_int(gp.w);
        const bool mask = a.excl_mask != nullptr;
        const unsigned emask = s_gm[il];
        const int e0 = mask ? 0 : a.excl_off[ai], e1 = mask ? 0 : a.excl_off[ai + 1];
        int ex[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) ex[e] = e0 + e < e1 ? a.excl_idx[e0 + e] : -1;
        int* const nbr_s = a.nbr + 4 * size_t(s);
        const unsigned stride = 4u * unsigned(a.nslots);
        const int2 run = s_gr[il];
        const int beg = max(run.x, w0) - w0;
        const int end = min(run.y, w0 + wn) - w0;
#define RELRES_SCAN(W, M)                                                                                  \
  scan_range<W, M>(s_pos, s_atom, beg, end, ai, px, py, pz, a.rl2, lx, ly, lz, emask, ex, e0, e1, a.excl_idx, \
                   a.excl_window, nbr_s, stride, a.cap, s_k[il])
        const int k = wrap ? (mask ? RELRES_SCAN(true, true) : RELRES_SCAN(true, false))
                           : (mask ? RELRES_SCAN(false, true) : RELRES_SCAN(false, false));
#undef RELRES_SCAN
        if (lane == 0) s_k[il] = k;
      }
    }
    __syncthreads();
    for (int il = threadIdx.x; il < ng; il += blockDim.x) {
      const int k = s_k[il];
      a.cnt[i0 + g0 + il] = min(k, a.cap);
      blk_max = max(blk_max, k);
      blk_tot += (unsigned long long)k;
    }
    __syncthreads();  // s_k is reused by the next group
  }
  // block statistics, then one atomic each
  blk_max = warp_max(blk_max);
  blk_tot = warp_sum(blk_tot);
  if (lane == 0) {
    atomicMax(&s_max, blk_max);
    atomicAdd(&s_tot, blk_tot);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(a.max_out, s_max);
    atomicAdd(a.total_out, s_tot);
    if (s_max > a.cap) atomicOr(a.flags, a.overflow_bit);
  }
  __syncthreads();  // shared memory is reused by the next cell
}

__global__ void __launch_bounds__(kListThreads) k_list(const unsigned* gate, ListArgs fg, ListArgs cg,
                                                       int ncell_cg) {
  if (gate_closed(gate)) return;
  const int ncell = ncell_cg + fg.g.ncell_full;
  for (int cb = blockIdx.x; cb < ncell; cb += gridDim.x) list_cell(fg, cg, ncell_cg, cb);
}

// grid-stride kernels: at most four blocks per SM (a closed gate then costs one small launch)
static int blocks_for(int n) {
  const int b = (n + kThreads - 1) / kThreads;
  return b < 1 ? 1 : (b > 152 * 4 ? 152 * 4 : b);
}

// ---- batches (relres_batch_step): the list rebuild of every replica whose
// displacement trigger fired, in seven launches for the whole batch.  After the
// drift, k_worklist lists those replicas and, per kernel class, the prefix
// sums of the blocks each of them takes in its own rebuild (the same counts as
// launch_rebuild / launch_lists); each batched kernel then walks the work
// items (replica, block) with a fixed grid, so a step in which few replicas
// rebuild costs seven short launches, and one in which none does, seven empty ones.

// Everything one replica's rebuild kernels take.
struct BuildArgs {
  int n, n_h_pack, hyb_mask, fp64;
  const unsigned* gate;
  const unsigned long long* xfx;
  const int* type;
  GridArgs gf, gc;
  int* cell_fg;
  int* slot_fg;
  int* cell_cg;
  int* slot_cg;
  unsigned* flags;
  int* perm_fg;
  int* perm_cg;
  int* rank_fg;
  int* rank_cg;
  int4* pos_fg;
  int4* pos_cg;
  Pos64* p64f;
  Pos64* p64c;
  int4* ref;
  DevState* st;
  ListArgs lfg, lcg;
  int ncell_cg;
};

enum { kRbBin = 0, kRbScanTiles, kRbScanAdd, kRbScatter, kRbSort, kRbPack, kRbList, kRbClasses };

// one block: wl[0] = number of rebuilding replicas, wl[1 .. nrep] their
// indices, then per class k the prefix sums pre_k[0 .. count] at
// wl + 1 + nrep + k (nrep + 1); nbt[k * nrep + r] = blocks of class k of replica r
__global__ void __launch_bounds__(1024) k_worklist(DevState* const* st, int nrep, const int* __restrict__ nbt,
                                                    int* __restrict__ wl, cudaGraphConditionalHandle any) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  int* rep = wl + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int r0 = 0; r0 < nrep; r0 += blockDim.x) {
    const int r = r0 + threadIdx.x;
    const int f = (r < nrep && (st[r]->flags & F_REBUILD)) ? 1 : 0;
    int incl = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int before = s_base;
    for (int w = 0; w < wid; ++w) before += s_warp[w];
    if (f) rep[before + incl - 1] = r;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < nw; ++w) s_base += s_warp[w];
    __syncthreads();
  }
  const int count = s_base;
  if (threadIdx.x == 0) {
    wl[0] = count;
    cudaGraphSetConditional(any, count > 0 ? 1u : 0u);  // the rebuild node runs iff a replica needs one
  }
  if (threadIdx.x < kRbClasses) {
    int* pre = wl + 1 + nrep + threadIdx.x * (nrep + 1);
    int acc = 0;
    for (int i = 0; i < count; ++i) {
      pre[i] = acc;
      acc += nbt[threadIdx.x * nrep + rep[i]];
    }
    pre[count] = acc;
  }
}

// Work item w of class K: replica *r, its block *b of *nb.
template <int K>
__device__ __forceinline__ int work_total(const int* wl, int nrep) {
  return wl[1 + nrep + K * (nrep + 1) + wl[0]];
}
template <int K>
__device__ __forceinline__ void work_item(const int* wl, const int* nbt, int nrep, int w, int* r, int* b, int* nb) {
  const int count = wl[0];
  const int* pre = wl + 1 + nrep + K * (nrep + 1);
  int lo = 0, hi = count - 1;  // the last i with pre[i] <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  *r = wl[1 + lo];
  *b = w - pre[lo];
  *nb = nbt[K * nrep + *r];
}

#define RELRES_BATCH_LOOP(K)                                       \
  const int total = work_total<K>(wl, nrep);                       \
  for (int w = blockIdx.x; w < total; w += gridDim.x) {            \
    int r, b, nb;                                                  \
    work_item<K>(wl, nbt, nrep, w, &r, &b, &nb);                   \
    const BuildArgs& sa = args[r];

#define RELRES_BATCH_END \
  }

__global__ void __launch_bounds__(kThreads, 6) k_bin_batch(const BuildArgs* __restrict__ args, const int* __restrict__ wl,
                            const int* __restrict__ nbt, int nrep) {
  RELRES_BATCH_LOOP(kRbBin)
  bin_body(b, nb, sa.n, sa.gate, sa.xfx, sa.type, sa.hyb_mask, sa.gf.n0, sa.gf.n1, sa.gf.n2, sa.gf.rank_of,
           sa.gf.count, sa.gc.valid, sa.gc.n0, sa.gc.n1, sa.gc.n2, sa.gc.rank_of, sa.gc.count, sa.cell_fg,
           sa.slot_fg, sa.cell_cg, sa.slot_cg, sa.flags);
  RELRES_BATCH_END
}

__global__ void __launch_bounds__(kScanTile / 4) k_scan_tiles_batch(const BuildArgs* __restrict__ args,
                                                                     const int* __restrict__ wl,
                                                                     const int* __restrict__ nbt, int nrep) {
  RELRES_BATCH_LOOP(kRbScanTiles)
  (void)nb;
  scan_tile_body(b, sa.gate, scan_grid(sa.gf), scan_grid(sa.gc), sa.st);
  RELRES_BATCH_END
}

__global__ void __launch_bounds__(kScanTile / 4) k_scan_add_batch(const BuildArgs* __restrict__ args,
                                                                   const int* __restrict__ wl,
                                                                   const int* __restrict__ nbt, int nrep) {
  RELRES_BATCH_LOOP(kRbScanAdd)
  (void)nb;
  scan_add_body(b, sa.gate, scan_grid(sa.gf), scan_grid(sa.gc));
  RELRES_BATCH_END
}

__global__ void __launch_bounds__(kThreads, 6) k_scatter_batch(const BuildArgs* __restrict__ args, const int* __restrict__ wl,
                                const int* __restrict__ nbt, int nrep) {
  RELRES_BATCH_LOOP(kRbScatter)
  scatter_body(b, nb, sa.n, sa.gate, sa.type, sa.hyb_mask, sa.gf.start, sa.gc.valid, sa.gc.start, sa.cell_fg,
               sa.slot_fg, sa.cell_cg, sa.slot_cg, sa.perm_fg, sa.perm_cg);
  RELRES_BATCH_END
}

__global__ void __launch_bounds__(kThreads, 6) k_sort_batch(const BuildArgs* __restrict__ args,
                                                         const int* __restrict__ wl, const int* __restrict__ nbt,
                                                         int nrep) {
  RELRES_BATCH_LOOP(kRbSort)
  sort_body(b, nb, sa.gate, sa.gf.ncell, sa.gf.start, sa.gc.valid ? sa.gc.ncell : 0, sa.gc.start, sa.perm_fg,
            sa.perm_cg);
  RELRES_BATCH_END
}

__global__ void __launch_bounds__(kThreads, 6) k_pack_batch(const BuildArgs* __restrict__ args, const int* __restrict__ wl,
                             const int* __restrict__ nbt, int nrep) {
  RELRES_BATCH_LOOP(kRbPack)
  pack_body(b, nb, sa.n, sa.n_h_pack, sa.gate, sa.xfx, sa.type, sa.perm_fg, sa.perm_cg, sa.rank_fg, sa.rank_cg,
            sa.pos_fg, sa.pos_cg, sa.p64f, sa.p64c, sa.fp64, sa.ref);
  RELRES_BATCH_END
}

__global__ void __launch_bounds__(kListThreads, 8) k_list_batch(const BuildArgs* __restrict__ args,
                                                             const int* __restrict__ wl,
                                                             const int* __restrict__ nbt, int nrep) {
  RELRES_BATCH_LOOP(kRbList)
  const int ncell = sa.ncell_cg + sa.lfg.g.ncell_full;
  for (int cb = b; cb < ncell; cb += nb) list_cell(sa.lfg, sa.lcg, sa.ncell_cg, cb);
  RELRES_BATCH_END
}

#undef RELRES_BATCH_LOOP
#undef RELRES_BATCH_END

// Arguments of one system's rebuild (binning and both lists), gated on `gate`.
static ListArgs list_args_fg(relres_ctx* c);
static bool list_args_cg(relres_ctx* c, ListArgs* cg, int* ncell_cg);

static BuildArgs build_args(relres_ctx* c, const unsigned* gate) {
  BuildArgs b{};
  b.gf = grid_args(c->gfg);
  b.gc = grid_args(c->gcg);
  if (!c->has_cg || c->n_h == 0) {
    b.gc = b.gf;  // stand-in pointers, never used
    b.gc.valid = 0;
  }
  b.n = c->n;
  b.n_h_pack = b.gc.valid ? c->n_h : 0;
  b.hyb_mask = c->hyb_mask;
  b.fp64 = c->fp64 ? 1 : 0;
  b.gate = gate;
  b.xfx = c->d_xfx;
  b.type = c->d_type;
  b.cell_fg = c->d_cell_fg;
  b.slot_fg = c->d_slot_fg;
  b.cell_cg = c->d_cell_cg;
  b.slot_cg = c->d_slot_cg;
  b.flags = &c->d_state->flags;
  b.perm_fg = c->d_perm_fg;
  b.perm_cg = c->d_perm_cg;
  b.rank_fg = c->d_rank_fg;
  b.rank_cg = c->d_rank_cg;
  b.pos_fg = c->d_pos_fg;
  b.pos_cg = c->d_pos_cg;
  b.p64f = c->fp64 ? c->d_pos_fg64 : static_cast<Pos64*>(c->d_dummy);
  b.p64c = c->fp64 ? c->d_pos_cg64 : static_cast<Pos64*>(c->d_dummy);
  b.ref = c->d_ref;
  b.st = c->d_state;
  b.lfg = list_args_fg(c);
  b.lcg = b.lfg;  // stand-in when there is no CG list (its blocks are not launched)
  b.ncell_cg = 0;
  list_args_cg(c, &b.lcg, &b.ncell_cg);
  return b;
}

// list-kernel blocks: persistent, one wave walks the cells (a closed gate costs one small launch)
static int list_blocks(const BuildArgs& b) { return std::min(b.ncell_cg + b.gf.ncell_full, 152 * 8); }
static int sort_cells_of(const BuildArgs& b) { return b.gf.ncell + (b.gc.valid ? b.gc.ncell : 0); }

cudaError_t launch_rebuild(relres_ctx* c, const unsigned* gate) {
  if (gate == nullptr) gate = c->d_open;
  const BuildArgs b = build_args(c, gate);
  const GridArgs& gf = b.gf;
  const GridArgs& gc = b.gc;
  const int nb = blocks_for(c->n);
  k_bin<<<nb, kThreads, 0, c->stream>>>(c->n, gate, c->d_xfx, c->d_type, c->hyb_mask, gf.n0, gf.n1,
                                        gf.n2, gf.rank_of, gf.count, gc.valid, gc.n0, gc.n1, gc.n2,
                                        gc.rank_of, gc.count, c->d_cell_fg, c->d_slot_fg, c->d_cell_cg,
                                        c->d_slot_cg, &c->d_state->flags);
  RELRES_LAUNCHED(c);
  const ScanGrid sf = scan_grid(gf), sc = scan_grid(gc);
  k_scan_tiles<<<sf.ntile + sc.ntile, kScanTile / 4, 0, c->stream>>>(gate, sf, sc, c->d_state);
  RELRES_LAUNCHED(c);
  k_scan_add<<<sf.ntile + sc.ntile, kScanTile / 4, 0, c->stream>>>(gate, sf, sc);
  RELRES_LAUNCHED(c);
  k_scatter<<<nb, kThreads, 0, c->stream>>>(c->n, gate, c->d_type, c->hyb_mask, gf.start, gc.valid, gc.start,
                                            c->d_cell_fg, c->d_slot_fg, c->d_cell_cg, c->d_slot_cg,
                                            c->d_perm_fg, c->d_perm_cg);
  RELRES_LAUNCHED(c);
  k_sort_cells<<<blocks_for(sort_cells_of(b)), kThreads, 0, c->stream>>>(
      gate, gf.ncell, gf.start, gc.valid ? gc.ncell : 0, gc.start, c->d_perm_fg, c->d_perm_cg);
  RELRES_LAUNCHED(c);
  k_pack<<<nb, kThreads, 0, c->stream>>>(c->n, b.n_h_pack, gate, c->d_xfx, c->d_type, c->d_perm_fg, c->d_perm_cg,
                                         c->d_rank_fg, c->d_rank_cg, c->d_pos_fg, c->d_pos_cg, b.p64f, b.p64c,
                                         b.fp64, c->d_ref);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t prepare_rebuild_batch(const std::vector<relres_ctx*>& cs, RebuildBatch* rb) {
  const int nr = int(cs.size());
  std::vector<BuildArgs> args(nr);
  std::vector<int> nbt(size_t(kRbClasses) * nr);
  for (int r = 0; r < nr; ++r) {
    relres_ctx* c = cs[r];
    args[r] = build_args(c, &c->d_state->flags);
    nbt[kRbBin * nr + r] = blocks_for(c->n);
    const int ntiles = args[r].gf.ntile + (args[r].gc.valid ? args[r].gc.ntile : 0);
    nbt[kRbScanTiles * nr + r] = ntiles;
    nbt[kRbScanAdd * nr + r] = ntiles;
    nbt[kRbScatter * nr + r] = blocks_for(c->n);
    nbt[kRbSort * nr + r] = blocks_for(sort_cells_of(args[r]));
    nbt[kRbPack * nr + r] = blocks_for(c->n);
    nbt[kRbList * nr + r] = list_blocks(args[r]);
  }
  const std::vector<int> off{0, nr};
  cudaError_t e = upload_batch(&rb->args, args.data(), sizeof(BuildArgs) * nr, off);
  if (e == cudaSuccess) e = upload_batch(&rb->nbt, nbt.data(), sizeof(int) * nbt.size(), off);
  const size_t wl_ints = 1 + size_t(nr) + size_t(kRbClasses) * (nr + 1);
  if (e == cudaSuccess && rb->wl_ints < wl_ints) {
    if (rb->d_wl) cudaFree(rb->d_wl);
    rb->d_wl = nullptr;
    rb->wl_ints = 0;
    e = cudaMalloc(&rb->d_wl, sizeof(int) * wl_ints);
    if (e == cudaSuccess) rb->wl_ints = wl_ints;
  }
  return e;
}

cudaError_t launch_worklist(cudaStream_t s, const RebuildBatch& rb, DevState* const* d_states, int nrep,
                            cudaGraphConditionalHandle any) {
  k_worklist<<<1, 1024, 0, s>>>(d_states, nrep, static_cast<const int*>(rb.nbt.d_args), rb.d_wl, any);
  return cudaGetLastError();
}

cudaError_t launch_rebuild_batch(cudaStream_t s, const RebuildBatch& rb, int nrep) {
  const auto* args = static_cast<const BuildArgs*>(rb.args.d_args);
  const int* nbt = static_cast<const int*>(rb.nbt.d_args);
  const int* wl = rb.d_wl;
  k_bin_batch<<<152 * 4, kThreads, 0, s>>>(args, wl, nbt, nrep);
  k_scan_tiles_batch<<<152, kScanTile / 4, 0, s>>>(args, wl, nbt, nrep);
  k_scan_add_batch<<<152, kScanTile / 4, 0, s>>>(args, wl, nbt, nrep);
  k_scatter_batch<<<152 * 4, kThreads, 0, s>>>(args, wl, nbt, nrep);
  k_sort_batch<<<152 * 4, kThreads, 0, s>>>(args, wl, nbt, nrep);
  k_pack_batch<<<152 * 4, kThreads, 0, s>>>(args, wl, nbt, nrep);
  k_list_batch<<<152 * 8, kListThreads, 0, s>>>(args, wl, nbt, nrep);
  return cudaGetLastError();
}

void free_rebuild_batch(RebuildBatch* rb) {
  free_batch(&rb->args);
  free_batch(&rb->nbt);
  if (rb->d_wl) cudaFree(rb->d_wl);
  *rb = RebuildBatch{};
}

// One thread: open the rebuild node of this step of a CUDA graph iff the
// displacement trigger fired (F_REBUILD is set by the drift kernel), and
// (with_prune) the pruning node iff either trigger fired.
__global__ void k_decide(const DevState* st, cudaGraphConditionalHandle h, cudaGraphConditionalHandle hp,
                         int with_prune) {
  const unsigned f = st->flags;
  cudaGraphSetConditional(h, (f & F_REBUILD) ? 1u : 0u);
  if (with_prune) cudaGraphSetConditional(hp, (f & (F_REBUILD | F_PRUNE)) ? 1u : 0u);
}

cudaError_t launch_decide(relres_ctx* c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle hp,
                          int with_prune) {
  k_decide<<<1, 1, 0, c->stream>>>(c->d_state, h, hp, with_prune);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

// ---- dynamic pruning (two-level lists).  The lists above hold every pair
// within the interaction cutoff + skin at the last build and stay valid until
// an atom has moved skin/2.  A pruning pass keeps, in list order, the entries
// whose current distance is below the interaction cutoff + delta; that list
// holds every interacting pair until an atom has moved delta/2 since the pass
// (two atoms then close in by at most delta), when the drift kernel sets
// F_PRUNE and the next step prunes again.  Since the kept entries keep their
// order and a dropped entry contributes exactly zero, the pair sums are
// bit-identical to those over the full lists (one thread per slot).

struct PruneList {
  int nslots;
  const int4* pos;  // sorted hi32 positions
  const int* nbr;   // full list (chunked layout)
  const int* cnt;
  int* nbr_in;      // pruned list, same layout and capacity
  int* cnt_in;
  float rp2;        // (interaction cutoff + delta + slack)^2
  unsigned long long* total;
};

struct PruneArgs {
  int nblk_cg;  // blocks [0, nblk_cg) prune the CG list, the rest the FG list
  PruneList fg, cg;
  float sx, sy, sz;
  const int* perm_fg;
  int4* ref_p;  // positions of this pass, caller order (written by the FG blocks)
  DevState* st;
};

constexpr int kPruneThreads = 256;

__device__ __forceinline__ int prune_slot(const PruneList& L, int s, float sx, float sy, float sz) {
  const int4 pi = L.pos[s];
  const int m = L.cnt[s];
  const int nch = (m + 3) >> 2;
  const int4* nb4 = reinterpret_cast<const int4*>(L.nbr) + s;
  int4* out4 = reinterpret_cast<int4*>(L.nbr_in) + s;
  int k = 0;
  int4 buf = make_int4(s, s, s, s);
  int4 jj = nch > 0 ? __ldcs(nb4) : buf;
  for (int ch = 0; ch < nch; ++ch) {
    int4 jn = jj;
    if (ch + 1 < nch) jn = __ldcs(nb4 + size_t(ch + 1) * L.nslots);
    const int rem = m - 4 * ch;  // >= 1
    const int j[4] = {jj.x, rem > 1 ? jj.y : s, rem > 2 ? jj.z : s, rem > 3 ? jj.w : s};
    int4 p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = __ldg(L.pos + j[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dx = dfix32(pi.x, p[q].x, sx), dy = dfix32(pi.y, p[q].y, sy), dz = dfix32(pi.z, p[q].z, sz);
      keep_entry((q == 0 || rem > q) && dx * dx + dy * dy + dz * dz < L.rp2, j[q], k, buf, out4, L.nslots);
    }
    jj = jn;
  }
  keep_tail(k, buf, out4, L.nslots);
  L.cnt_in[s] = k;
  return k;
}

__global__ void __launch_bounds__(kPruneThreads) k_prune(const unsigned* gate, PruneArgs a) {
  if (gate_closed(gate, F_REBUILD | F_PRUNE)) return;
  const bool is_cg = int(blockIdx.x) < a.nblk_cg;
  const int blk = is_cg ? blockIdx.x : blockIdx.x - a.nblk_cg;
  const int s = blk * kPruneThreads + threadIdx.x;
  unsigned long long kept = 0ull;
  if (is_cg) {
    if (s < a.cg.nslots) kept = prune_slot(a.cg, s, a.sx, a.sy, a.sz);
  } else if (s < a.fg.nslots) {
    kept = prune_slot(a.fg, s, a.sx, a.sy, a.sz);
    a.ref_p[a.perm_fg[s]] = a.fg.pos[s];
  }
  __shared__ unsigned long long sh[kPruneThreads / 32];
  kept = warp_sum(kept);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = kept;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0ull;
    for (int w = 0; w < kPruneThreads / 32; ++w) t += sh[w];
    atomicAdd(is_cg ? a.cg.total : a.fg.total, t);
    if (blockIdx.x == 0) atomicAdd(&a.st->n_prunes, 1ull);
  }
}

cudaError_t launch_prune(relres_ctx* c, const unsigned* gate) {
  if (!c->prune_on) return cudaSuccess;
  if (gate == nullptr) gate = c->d_open;
  const float s0 = float(c->box[0] / 4294967296.0), s1 = float(c->box[1] / 4294967296.0),
              s2 = float(c->box[2] / 4294967296.0);
  DevState* st = c->d_state;
  const double rf = c->rlist_fg_cut + c->prune_delta + kPruneSlack;
  PruneArgs a;
  a.fg = PruneList{c->n, c->d_pos_fg, c->d_nbr_fg, c->d_cnt_fg, c->d_nbr_fg_in, c->d_cnt_fg_in,
                   float(rf * rf), &st->tot_in_fg};
  a.cg = a.fg;  // stand-in when there is no CG list (no CG blocks are launched)
  a.nblk_cg = 0;
  if (c->has_cg && c->n_h > 0) {
    const double rc = c->rlist_cg_cut + c->prune_delta + kPruneSlack;
    a.cg = PruneList{c->n_h, c->d_pos_cg, c->d_nbr_cg, c->d_cnt_cg, c->d_nbr_cg_in, c->d_cnt_cg_in,
                     float(rc * rc), &st->tot_in_cg};
    a.nblk_cg = (c->n_h + kPruneThreads - 1) / kPruneThreads;
  }
  a.sx = s0;
  a.sy = s1;
  a.sz = s2;
  a.perm_fg = c->d_perm_fg;
  a.ref_p = c->d_ref_p;
  a.st = st;
  const int nb = a.nblk_cg + (c->n + kPruneThreads - 1) / kPruneThreads;
  k_prune<<<nb, kPruneThreads, 0, c->stream>>>(gate, a);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

static ListArgs list_args_fg(relres_ctx* c) {
  const float s0 = float(c->box[0] / 4294967296.0), s1 = float(c->box[1] / 4294967296.0),
              s2 = float(c->box[2] / 4294967296.0);
  DevState* st = c->d_state;
  const double rf = c->rlist_fg_cut + c->prm.skin;
  return ListArgs{c->n, c->d_pos_fg, c->d_perm_fg, grid_args(c->gfg), s0, s1, s2, float(rf * rf),
                  c->d_excl_off, c->d_excl_idx, c->excl_window, c->cap_fg, c->d_nbr_fg, c->d_cnt_fg,
                  &st->max_fg, &st->tot_fg, &st->flags, F_OVERFLOW_FG, c->d_excl_mask};
}

// the CG list's arguments and cells; false (arguments untouched) without a CG list
static bool list_args_cg(relres_ctx* c, ListArgs* cg, int* ncell_cg) {
  if (!(c->has_cg && c->n_h > 0)) return false;
  const float s0 = float(c->box[0] / 4294967296.0), s1 = float(c->box[1] / 4294967296.0),
              s2 = float(c->box[2] / 4294967296.0);
  DevState* st = c->d_state;
  const double rc = c->rlist_cg_cut + c->skin_cg;
  *cg = ListArgs{c->n_h, c->d_pos_cg, c->d_perm_cg, grid_args(c->gcg), s0, s1, s2, float(rc * rc),
                 c->d_excl_off, c->d_excl_idx, c->excl_window, c->cap_cg, c->d_nbr_cg, c->d_cnt_cg,
                 &st->max_cg, &st->tot_cg, &st->flags, F_OVERFLOW_CG, c->d_excl_mask};
  *ncell_cg = c->gcg.ncell_full;
  return true;
}

cudaError_t launch_lists(relres_ctx* c, const unsigned* gate) {
  if (gate == nullptr) gate = c->d_open;
  const ListArgs fg = list_args_fg(c);
  ListArgs cg = fg;  // stand-in when there is no CG list (its blocks are not launched)
  int ncell_cg = 0;
  list_args_cg(c, &cg, &ncell_cg);
  // persistent: one wave of blocks walks the full cells (a closed gate costs one small launch)
  const int nb = std::min(ncell_cg + c->gfg.ncell_full, 152 * 8);
  k_list<<<nb, kListThreads, 0, c->stream>>>(gate, fg, cg, ncell_cg);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

}  // namespace relres
