// Backward pass of the RelRes pair interaction (the differentiable form of
// Eq. 20, Section 2.5): gradients of a scalar L(E, F) of the pair energy E
// and the pair forces F with respect to the positions and to the LJ
// parameters, given gE = dL/dE and g_i = dL/dF_i.
//
// Every smoothing coefficient (Eq. 17, Eq. 18) and shift (Eq. 19) is linear
// in the potential, so for each type pair and each part of the exact FG/CG
// split  u~ = C12 phi12(r) - C6 phi6(r)  with C12 = 4 eps sig^12,
// C6 = 4 eps sig^6 and phik the same construction applied to r^-k
// (BasisTab).  Hence
//   dL/dC12 = gE S12 + T12,   dL/dC6 = -(gE S6 + T6),
//   S_k = sum over pairs of phik(r),  T_k = sum_i g_i . sum_j (-phik'(r) rhat_ij),
//   dL/dx_i = gE sum_j u~'(r) rhat_ij - sum_j h_ij (g_i - g_j),
//   h_ij = u~''(r) rhat rhat^T + (u~'(r)/r) (I - rhat rhat^T)
// (the second term is the Hessian-vector product of E with g).  The C2
// smoothing of the paper makes u~'' well defined in every region.
//
// One launch walks both lists (CG blocks first) like the force kernel; the
// lists are those of the last force evaluation (nothing of the forward pass
// is stored besides them).  Per-type-pair sums are kept per thread in
// registers (the atom's own type is fixed, the partner's type selects the
// accumulator), reduced per block in shared memory and added to FP64 totals
// with atomics.
#include "common.cuh"

namespace relres {

template <typename R>
using GVec = typename std::conditional<std::is_same<R, float>::value, float4, double>::type;
template <typename R>
using GPos = typename std::conditional<std::is_same<R, float>::value, int4, Pos64>::type;

__device__ __forceinline__ void ld3(const float4* a, int i, float v[3]) {
  const float4 q = a[i];
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
}
__device__ __forceinline__ void ld3(const double* a, int i, double v[3]) {
  v[0] = a[3 * i];
  v[1] = a[3 * i + 1];
  v[2] = a[3 * i + 2];
}
__device__ __forceinline__ void st3(float4* a, int i, const float v[3]) { a[i] = make_float4(v[0], v[1], v[2], 0.f); }
__device__ __forceinline__ void st3(double* a, int i, const double v[3]) {
  a[3 * i] = v[0];
  a[3 * i + 1] = v[1];
  a[3 * i + 2] = v[2];
}
__device__ __forceinline__ void diff3(const int4& a, const int4& b, float sx, float sy, float sz, float d[3]) {
  d[0] = dfix32(a.x, b.x, sx);
  d[1] = dfix32(a.y, b.y, sy);
  d[2] = dfix32(a.z, b.z, sz);
}
__device__ __forceinline__ void diff3(const Pos64& a, const Pos64& b, double sx, double sy, double sz,
                                      double d[3]) {
  d[0] = dfix64(a.x, b.x, sx);
  d[1] = dfix64(a.y, b.y, sy);
  d[2] = dfix64(a.z, b.z, sz);
}
__device__ __forceinline__ int gtype(const int4& p) { return p.w; }
__device__ __forceinline__ int gtype(const Pos64& p) { return int(p.t); }

// f, f', f'' of the quartic Eq. 16 at d
template <typename R>
__device__ __forceinline__ void poly3(const R (&g)[5], R d, R& f, R& f1, R& f2) {
  f = (((g[4] * d + g[3]) * d + g[2]) * d + g[1]) * d + g[0];
  f1 = ((R(4) * g[4] * d + R(3) * g[3]) * d + R(2) * g[2]) * d + g[1];
  f2 = (R(12) * g[4] * d + R(6) * g[3]) * d + R(2) * g[2];
}

// phi, phi', phi'' of both bases (b = 0: r^-12, b = 1: r^-6) for one part.
template <typename R, bool CG>
__device__ __forceinline__ void basis(const BasisTab<R>& T, R r, R ri, R (&p)[2], R (&p1)[2], R (&p2)[2]) {
  const R r2i = ri * ri;
  const R v6 = r2i * r2i * r2i;
  const R v[2] = {v6 * v6, v6};
  const R kk[2] = {R(12), R(6)};
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (!CG) {
      if (r < T.rsm) {
        p[b] = v[b] - T.fg_sh[b];
        p1[b] = -kk[b] * v[b] * ri;
        p2[b] = kk[b] * (kk[b] + R(1)) * v[b] * r2i;
      } else {
        poly3<R>(T.fg[b], r - T.rsm, p[b], p1[b], p2[b]);
        p[b] -= T.fg_sh[b];
      }
    } else {
      if (r < T.rsm) {
        p[b] = T.on[b][0] - T.gam[b];
        p1[b] = R(0);
        p2[b] = R(0);
      } else if (r < T.rsp) {
        poly3<R>(T.on[b], r - T.rsm, p[b], p1[b], p2[b]);
        p[b] -= T.gam[b];
      } else if (r < T.rcm) {
        p[b] = v[b] - T.gam[b];
        p1[b] = -kk[b] * v[b] * ri;
        p2[b] = kk[b] * (kk[b] + R(1)) * v[b] * r2i;
      } else {
        poly3<R>(T.off[b], r - T.rcm, p[b], p1[b], p2[b]);
        p[b] -= T.gam[b];
      }
    }
  }
}

template <typename R>
struct GradWalk {
  int nslots;
  const GPos<R>* pos;
  const int* nbr;
  const int* cnt;
  const int* perm;
  const GVec<R>* g;  // dL/dF in this list's slot order
  GVec<R>* gx;       // dL/dx of this list's part, caller order
};

template <typename R>
struct GradLaunch {
  int nblk_cg;
  GradWalk<R> fg, cg;
  const BasisTab<R>* tab;
  int nt;
  R sx, sy, sz;
  R g_energy;
  double* gc;  // [nt*nt][4]: dL/dC12_FG, dL/dC6_FG, dL/dC12_CG, dL/dC6_CG
};

template <typename R, bool CG>
__device__ __forceinline__ void grad_walk(const GradWalk<R>& W, int blk, const BasisTab<R>* tab,
                                          const GradLaunch<R>& a, double* s_gc) {
  const int s = blk * blockDim.x + threadIdx.x;
  R acc12[RELRES_MAX_TYPES], acc6[RELRES_MAX_TYPES];
#pragma unroll
  for (int t = 0; t < RELRES_MAX_TYPES; ++t) acc12[t] = acc6[t] = R(0);
  int ti = 0;
  if (s < W.nslots) {
    const auto pi = W.pos[s];
    ti = gtype(pi);
    R gi[3], gx[3] = {R(0), R(0), R(0)};
    ld3(W.g, s, gi);
    const int m = W.cnt[s];
    for (int k = 0; k < m; ++k) {
      const int j = W.nbr[((size_t(k >> 2) * W.nslots + s) << 2) + (k & 3)];
      const auto pj = W.pos[j];
      const int tj = gtype(pj);
      const BasisTab<R>& T = tab[ti * a.nt + tj];
      R d[3];
      diff3(pi, pj, a.sx, a.sy, a.sz, d);
      const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const R rcut = CG ? T.rcp : T.rsp;
      if (!(r2 < rcut * rcut)) continue;
      const R r = sqrt(r2);
      const R ri = R(1) / r;
      R p[2], p1[2], p2[2];
      basis<R, CG>(T, r, ri, p, p1, p2);
      const R c12 = CG ? T.c12c : T.c12f, c6 = CG ? T.c6c : T.c6f;
      const R u1 = c12 * p1[0] - c6 * p1[1];
      const R u2 = c12 * p2[0] - c6 * p2[1];
      R gj[3];
      ld3(W.g, j, gj);
      R rh[3], w[3];
      R rw = R(0), gir = R(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        rh[q] = d[q] * ri;
        w[q] = gi[q] - gj[q];
        rw += rh[q] * w[q];
        gir += gi[q] * rh[q];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q)
        gx[q] += a.g_energy * u1 * rh[q] - (u2 * rw * rh[q] + u1 * ri * (w[q] - rw * rh[q]));
      const R e12 = R(0.5) * a.g_energy * p[0] - p1[0] * gir;
      const R e6 = R(0.5) * a.g_energy * p[1] - p1[1] * gir;
#pragma unroll
      for (int t = 0; t < RELRES_MAX_TYPES; ++t) {
        acc12[t] += t == tj ? e12 : R(0);
        acc6[t] += t == tj ? e6 : R(0);
      }
    }
    st3(W.gx, W.perm[s], gx);
  }
  // per-type-pair sums: shared-memory FP64 atomics per block, then global
  if (s < W.nslots) {
#pragma unroll
    for (int t = 0; t < RELRES_MAX_TYPES; ++t) {
      if (t < a.nt && acc12[t] != R(0)) atomicAdd(&s_gc[(ti * a.nt + t) * 2], double(acc12[t]));
      if (t < a.nt && acc6[t] != R(0)) atomicAdd(&s_gc[(ti * a.nt + t) * 2 + 1], -double(acc6[t]));
    }
  }
}

template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_pair_grad(GradLaunch<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = a.nt * a.nt;
  BasisTab<R>* tab = reinterpret_cast<BasisTab<R>*>(smem_raw);
  double* s_gc = reinterpret_cast<double*>(smem_raw + ((sizeof(BasisTab<R>) * nrow + 15) / 16) * 16);
  {
    const int words = nrow * int(sizeof(BasisTab<R>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(a.tab);
    int* dst = reinterpret_cast<int*>(tab);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  for (int q = threadIdx.x; q < 2 * nrow; q += blockDim.x) s_gc[q] = 0.0;
  __syncthreads();
  const bool cg = int(blockIdx.x) < a.nblk_cg;
  if (cg)
    grad_walk<R, true>(a.cg, blockIdx.x, tab, a, s_gc);
  else
    grad_walk<R, false>(a.fg, blockIdx.x - a.nblk_cg, tab, a, s_gc);
  __syncthreads();
  const int off = cg ? 2 : 0;
  for (int q = threadIdx.x; q < 2 * nrow; q += blockDim.x)
    if (s_gc[q] != 0.0) atomicAdd(&a.gc[(q >> 1) * 4 + off + (q & 1)], s_gc[q]);
}

// dL/dF (caller order, FP64) into one list's slot order
template <typename R>
__global__ void k_gather_g(int nslots, const int* __restrict__ perm, const double* __restrict__ g,
                           GVec<R>* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
    const int i = perm[s];
    const R v[3] = {R(g[3 * i]), R(g[3 * i + 1]), R(g[3 * i + 2])};
    st3(out, s, v);
  }
}

// dL/dx = FG part + CG part (hybrids), caller order, FP64 out
template <typename R>
__global__ void k_sum_gx(int n, const GVec<R>* __restrict__ gx_fg, const GVec<R>* __restrict__ gx_cg,
                         int with_cg, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    R a[3], b[3] = {R(0), R(0), R(0)};
    ld3(gx_fg, i, a);
    if (with_cg) ld3(gx_cg, i, b);
    out[3 * i] = double(a[0]) + double(b[0]);
    out[3 * i + 1] = double(a[1]) + double(b[1]);
    out[3 * i + 2] = double(a[2]) + double(b[2]);
  }
}

static int grid_for(int n) {
  const int b = (n + kThreads - 1) / kThreads;
  return b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b);
}

template <typename R>
static cudaError_t launch_grad_t(relres_ctx* c, const double* d_grad_forces, double g_energy, double* d_grad_pos) {
  using V = GVec<R>;
  const bool do_cg = c->has_cg && c->n_h > 0;
  const double* g = d_grad_forces ? d_grad_forces : static_cast<const double*>(c->d_zero_n3);
  V* gfg = static_cast<V*>(c->d_g_fg);
  V* gcg = static_cast<V*>(c->d_g_cg);
  V* xfg = static_cast<V*>(c->d_gx_fg);
  V* xcg = static_cast<V*>(c->d_gx_cg);
  k_gather_g<R><<<grid_for(c->n), kThreads, 0, c->stream>>>(c->n, c->d_perm_fg, g, gfg);
  RELRES_LAUNCHED(c);
  if (do_cg) {
    k_gather_g<R><<<grid_for(c->n_h), kThreads, 0, c->stream>>>(c->n_h, c->d_perm_cg, g, gcg);
    RELRES_LAUNCHED(c);
  }
  const double unit = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  GradLaunch<R> a{};
  a.sx = R(c->box[0] / unit);
  a.sy = R(c->box[1] / unit);
  a.sz = R(c->box[2] / unit);
  a.nt = c->n_types;
  a.tab = static_cast<const BasisTab<R>*>(c->d_basis);
  a.g_energy = R(g_energy);
  a.gc = c->d_gc;
  const GPos<R>* pfg;
  const GPos<R>* pcg;
  if constexpr (std::is_same<R, float>::value) {
    pfg = c->d_pos_fg;
    pcg = c->d_pos_cg;
  } else {
    pfg = c->d_pos_fg64;
    pcg = c->d_pos_cg64;
  }
  a.fg = GradWalk<R>{c->n, pfg, walk_nbr_fg(c), walk_cnt_fg(c), c->d_perm_fg, gfg, xfg};
  a.cg = do_cg ? GradWalk<R>{c->n_h, pcg, walk_nbr_cg(c), walk_cnt_cg(c), c->d_perm_cg, gcg, xcg} : a.fg;
  // small systems: 64-thread blocks, so that the launch covers every SM
  const int bs = c->n < 200000 ? 64 : kThreads;
  const int nb_fg = (c->n + bs - 1) / bs;
  const int nb_cg = do_cg ? (c->n_h + bs - 1) / bs : 0;
  a.nblk_cg = nb_cg;
  const int nrow = c->n_types * c->n_types;
  const size_t smem = ((sizeof(BasisTab<R>) * nrow + 15) / 16) * 16 + sizeof(double) * 2 * nrow;
  const cudaError_t ez = cudaMemsetAsync(c->d_gc, 0, sizeof(double) * 4 * nrow, c->stream);
  if (ez != cudaSuccess) return ez;
  if (bs == 64)
    k_pair_grad<R, 64><<<nb_cg + nb_fg, 64, smem, c->stream>>>(a);
  else
    k_pair_grad<R, kThreads><<<nb_cg + nb_fg, kThreads, smem, c->stream>>>(a);
  RELRES_LAUNCHED(c);
  if (d_grad_pos) {
    k_sum_gx<R><<<grid_for(c->n), kThreads, 0, c->stream>>>(c->n, xfg, xcg, do_cg ? 1 : 0, d_grad_pos);
    RELRES_LAUNCHED(c);
  }
  return cudaGetLastError();
}

cudaError_t launch_pair_grad(relres_ctx* c, const double* d_grad_forces, double g_energy, double* d_grad_pos) {
  return c->fp64 ? launch_grad_t<double>(c, d_grad_forces, g_energy, d_grad_pos)
                 : launch_grad_t<float>(c, d_grad_forces, g_energy, d_grad_pos);
}

}  // namespace relres
