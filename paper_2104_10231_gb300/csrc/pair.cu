// RelRes pair kernels: Eq. 20 of the paper (Section 2.5) over the two lists.
//
// The potential is evaluated split exactly into an FG part (on the FG list:
// every atom, partners within r_s+) and a CG part (on the CG list: hybrid
// sites, partners within r_c+), see PairTab in relres_internal.h.  Forces
// never depend on a shift constant, so the split changes nothing but which
// list carries which term.
//
// One thread owns one sorted slot and walks its full list: per entry a
// coalesced 4-byte index load, one 16-byte gather of the partner's packed
// position (L1/L2-resident thanks to the Morton cell order), an exact
// wrapped integer difference converted to FP32, and the region test.  The
// owner accumulates its force in registers and writes it once (no atomics).
// Energy and virial are optional per launch (EV template); they are reduced
// per block (warp shuffles, then shared memory) and written as 64-bit fixed
// point partial sums.  The FP64 variant (R = double) reads 64-bit fixed-point
// positions and computes every term in double.
#include "common.cuh"

namespace relres {

template <typename R>
struct PosOf;
template <>
struct PosOf<float> {
  using T = int4;
};
template <>
struct PosOf<double> {
  using T = Pos64;
};

__device__ __forceinline__ void delta(const int4& a, const int4& b, float sx, float sy, float sz,
                                      float& dx, float& dy, float& dz) {
  dx = dfix32(a.x, b.x, sx);
  dy = dfix32(a.y, b.y, sy);
  dz = dfix32(a.z, b.z, sz);
}
__device__ __forceinline__ void delta(const Pos64& a, const Pos64& b, double sx, double sy,
                                      double sz, double& dx, double& dy, double& dz) {
  dx = dfix64(a.x, b.x, sx);
  dy = dfix64(a.y, b.y, sy);
  dz = dfix64(a.z, b.z, sz);
}
__device__ __forceinline__ int ptype(const int4& p) { return p.w; }
__device__ __forceinline__ int ptype(const Pos64& p) { return int(p.t); }

__device__ __forceinline__ int4 load_pos(const int4* p, int j) { return __ldg(p + j); }
__device__ __forceinline__ Pos64 load_pos(const Pos64* p, int j) { return p[j]; }

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

__device__ __forceinline__ void store_force(float4* f, int i, float x, float y, float z) {
  f[i] = make_float4(x, y, z, 0.f);
}
__device__ __forceinline__ void store_force(double* f, int i, double x, double y, double z) {
  f[3 * i] = x;
  f[3 * i + 1] = y;
  f[3 * i + 2] = z;
}

template <typename R>
struct PairArgs {
  int nslots;
  const typename PosOf<R>::T* pos;
  const int* nbr;
  const int* cnt;
  const int* perm;
  const PairTab<R>* tab;
  int nt;
  R sx, sy, sz;
  typename std::conditional<std::is_same<R, float>::value, float4, double>::type* f_out;
  long long* partial;  // [gridDim.x][kNQ]
  const DevState* st;
};

// FG part for one entry.  Returns false outside r_s+.
template <typename R, bool EV>
__device__ __forceinline__ bool fg_term(const PairTab<R>& T, R r2, R& fr, R& ep) {
  if (!(r2 < T.rsp2)) return false;
  if (r2 < T.rsm2) {
    const R r2i = recip(r2);
    const R r6i = r2i * r2i * r2i;
    fr = r6i * (T.f12f * r6i - T.f6f) * r2i;
    if (EV) ep = r6i * (T.c12f * r6i - T.c6f) - T.e_fg_shift;
  } else {
    const R ri = rsq(r2);
    const R d = r2 * ri - T.rsm;
    const R fp = ((T.fgd[3] * d + T.fgd[2]) * d + T.fgd[1]) * d + T.fgd[0];
    fr = -fp * ri;
    if (EV) ep = ((((T.fg[4] * d + T.fg[3]) * d + T.fg[2]) * d + T.fg[1]) * d + T.fg[0]) - T.e_fg_shift;
  }
  return true;
}

// CG part for one entry.  Returns false outside r_c+.
template <typename R, bool EV>
__device__ __forceinline__ bool cg_term(const PairTab<R>& T, R r2, R& fr, R& ep) {
  if (!(r2 < T.rcp2)) return false;
  if (r2 < T.rsm2) {  // constant: f_{s+}(0) - Gamma_{c-}, no force
    fr = R(0);
    if (EV) ep = T.e_cg_close;
    return true;
  }
  const R ri = rsq(r2);
  if (r2 < T.rsp2) {  // switching on
    const R d = r2 * ri - T.rsm;
    const R d2 = d * d;
    fr = -(d2 * (T.ond4 * d + T.ond3)) * ri;
    if (EV) ep = T.on0 + d2 * d * (T.on4 * d + T.on3) - T.gam_cm;
  } else if (r2 < T.rcm2) {  // CG LJ
    const R r2i = ri * ri;
    const R r6i = r2i * r2i * r2i;
    fr = r6i * (T.f12c * r6i - T.f6c) * r2i;
    if (EV) ep = r6i * (T.c12c * r6i - T.c6c) - T.gam_cm;
  } else {  // switching off
    const R d = r2 * ri - T.rcm;
    const R fp = ((T.cgod[3] * d + T.cgod[2]) * d + T.cgod[1]) * d + T.cgod[0];
    fr = -fp * ri;
    if (EV) ep = ((((T.cgo[4] * d + T.cgo[3]) * d + T.cgo[2]) * d + T.cgo[1]) * d + T.cgo[0]) - T.gam_cm;
  }
  return true;
}

template <typename R, bool CG, bool EV>
__device__ __forceinline__ void pair_body(PairArgs<R> a, const PairTab<R>* tab) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  R fx = R(0), fy = R(0), fz = R(0);
  R acc[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q] = R(0);
  if (s < a.nslots) {
    const auto pi = a.pos[s];
    const PairTab<R>* trow = tab + ptype(pi) * a.nt;
    const int m = a.cnt[s];
    const int* nb = a.nbr + s;
    for (int k = 0; k < m; ++k) {
      const int j = __ldg(nb + (size_t)k * a.nslots);
      const auto pj = load_pos(a.pos, j);
      R dx, dy, dz;
      delta(pi, pj, a.sx, a.sy, a.sz, dx, dy, dz);
      const R r2 = dx * dx + dy * dy + dz * dz;
      const PairTab<R>& T = trow[ptype(pj)];
      R fr, ep;
      const bool hit = CG ? cg_term<R, EV>(T, r2, fr, ep) : fg_term<R, EV>(T, r2, fr, ep);
      if (hit) {
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        if (EV) {
          acc[0] += ep;
          acc[1] += fr * dx * dx;
          acc[2] += fr * dy * dy;
          acc[3] += fr * dz * dz;
          acc[4] += fr * dx * dy;
          acc[5] += fr * dx * dz;
          acc[6] += fr * dy * dz;
        }
      }
    }
    store_force(a.f_out, a.perm[s], fx, fy, fz);
  }
  if (EV) {
    __shared__ R sh[(kThreads / 32) * kNQ];
    block_sum<R, kNQ>(acc, sh);
    if (threadIdx.x == 0) {
      // full lists: every pair was visited from both ends
#pragma unroll
      for (int q = 0; q < kNQ; ++q) a.partial[blockIdx.x * kNQ + q] = to_fix_sum(0.5 * double(acc[q]));
    }
  }
}

template <typename R, bool CG>
__global__ void __launch_bounds__(kThreads) k_pair(PairArgs<R> a, int ev_mode) {
  extern __shared__ unsigned char smem_raw[];
  PairTab<R>* tab = reinterpret_cast<PairTab<R>*>(smem_raw);
  const int nrow = a.nt * a.nt;
  const int words = nrow * int(sizeof(PairTab<R>) / sizeof(int));
  const int* src = reinterpret_cast<const int*>(a.tab);
  int* dst = reinterpret_cast<int*>(smem_raw);
  for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  const bool ev = ev_mode == 1 || (ev_mode == 2 && a.st->ev);
  if (ev)
    pair_body<R, CG, true>(a, tab);
  else
    pair_body<R, CG, false>(a, tab);
}

template <typename R>
static cudaError_t launch_pairs_t(relres_ctx* c, int ev_mode, int which) {
  using F = typename std::conditional<std::is_same<R, float>::value, float4, double>::type;
  const R sx = R(c->box[0] / (std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0));
  const R sy = R(c->box[1] / (std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0));
  const R sz = R(c->box[2] / (std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0));
  const size_t smem = sizeof(PairTab<R>) * c->n_types * c->n_types;
  const typename PosOf<R>::T* pfg;
  const typename PosOf<R>::T* pcg;
  if constexpr (std::is_same<R, float>::value) {
    pfg = c->d_pos_fg;
    pcg = c->d_pos_cg;
  } else {
    pfg = c->d_pos_fg64;
    pcg = c->d_pos_cg64;
  }
  if (which & 1) {
    PairArgs<R> a{c->n, pfg, c->d_nbr_fg, c->d_cnt_fg, c->d_perm_fg,
                  static_cast<const PairTab<R>*>(c->d_tab), c->n_types, sx, sy, sz,
                  static_cast<F*>(c->d_f_fg), c->d_part_fg, c->d_state};
    k_pair<R, false><<<(c->n + kThreads - 1) / kThreads, kThreads, smem, c->stream>>>(a, ev_mode);
    RELRES_LAUNCHED(c);
  }
  if ((which & 2) && c->has_cg && c->n_h > 0) {
    PairArgs<R> a{c->n_h, pcg, c->d_nbr_cg, c->d_cnt_cg, c->d_perm_cg,
                  static_cast<const PairTab<R>*>(c->d_tab), c->n_types, sx, sy, sz,
                  static_cast<F*>(c->d_f_cg), c->d_part_cg, c->d_state};
    k_pair<R, true><<<(c->n_h + kThreads - 1) / kThreads, kThreads, smem, c->stream>>>(a, ev_mode);
    RELRES_LAUNCHED(c);
  }
  return cudaGetLastError();
}

cudaError_t launch_pairs(relres_ctx* c, int ev_mode, int which) {
  return c->fp64 ? launch_pairs_t<double>(c, ev_mode, which) : launch_pairs_t<float>(c, ev_mode, which);
}

}  // namespace relres
