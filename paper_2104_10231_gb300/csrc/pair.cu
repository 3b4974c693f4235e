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
  const PairTab<double>* tabd;  // FP64 table: energies of the FP32 path are evaluated in FP64
  int nt;
  R sx, sy, sz;
  double sxd, syd, szd;  // L / 2^32 (FP32 path) for the FP64 energy
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

__device__ __forceinline__ double dfix32d(int a, int b, double scale) {
  return double(int(unsigned(a) - unsigned(b))) * scale;
}

// One slot's walk over its list.  Energies: FP32 path -> FP64 evaluation from
// the exact coordinate differences (energy steps only); FP64 path -> FP64.
template <typename R, bool CG, bool EV>
__device__ __forceinline__ void pair_body(int nslots, const typename PosOf<R>::T* __restrict__ pos,
                                          const int* __restrict__ nbr, const int* __restrict__ cnt,
                                          const int* __restrict__ perm, const PairTab<R>* tab,
                                          const PairTab<double>* tabd, int nt, R sx, R sy, R sz,
                                          double sxd, double syd, double szd,
                                          typename std::conditional<std::is_same<R, float>::value,
                                                                    float4, double>::type* f_out,
                                          long long* partial) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  R fx = R(0), fy = R(0), fz = R(0);
  double e_acc = 0.0;
  R acc[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q] = R(0);
  if (s < nslots) {
    const auto pi = pos[s];
    const PairTab<R>* trow = tab + ptype(pi) * nt;
    const PairTab<double>* trowd = tabd + ptype(pi) * nt;
    const int m = cnt[s];
    const int* nb = nbr + s;
    for (int k = 0; k < m; ++k) {
      const int j = __ldg(nb + (size_t)k * nslots);
      const auto pj = load_pos(pos, j);
      R dx, dy, dz;
      delta(pi, pj, sx, sy, sz, dx, dy, dz);
      const R r2 = dx * dx + dy * dy + dz * dz;
      const PairTab<R>& T = trow[ptype(pj)];
      R fr, ep;
      const bool hit = CG ? cg_term<R, EV>(T, r2, fr, ep) : fg_term<R, EV>(T, r2, fr, ep);
      if (hit) {
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        if (EV) {
          if constexpr (std::is_same<R, double>::value) acc[0] += ep;
          acc[1] += fr * dx * dx;
          acc[2] += fr * dy * dy;
          acc[3] += fr * dz * dz;
          acc[4] += fr * dx * dy;
          acc[5] += fr * dx * dz;
          acc[6] += fr * dy * dz;
        }
      }
      if constexpr (EV && std::is_same<R, float>::value) {
        const double ex = dfix32d(pi.x, pj.x, sxd), ey = dfix32d(pi.y, pj.y, syd),
                     ez = dfix32d(pi.z, pj.z, szd);
        double frd, epd;
        const PairTab<double>& Td = trowd[ptype(pj)];
        if (CG ? cg_term<double, true>(Td, ex * ex + ey * ey + ez * ez, frd, epd)
               : fg_term<double, true>(Td, ex * ex + ey * ey + ez * ez, frd, epd))
          e_acc += epd;
      }
    }
    store_force(f_out, perm[s], fx, fy, fz);
  }
  if (EV) {
    // per-thread sums are R (FP64 for the energy); the block sum is taken in FP64
    double accd[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) accd[q] = double(acc[q]);
    if constexpr (std::is_same<R, float>::value) accd[0] = e_acc;
    __shared__ double sh[(kThreads / 32) * kNQ];
    block_sum<double, kNQ>(accd, sh);
    if (threadIdx.x == 0) {
      // full lists: every pair was visited from both ends
#pragma unroll
      for (int q = 0; q < kNQ; ++q) partial[blockIdx.x * kNQ + q] = to_fix_sum(0.5 * accd[q]);
    }
  }
}

template <typename R, bool CG>
__global__ void __launch_bounds__(kThreads) k_pair(PairArgs<R> a, int ev_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = a.nt * a.nt;
  PairTab<R>* tab = reinterpret_cast<PairTab<R>*>(smem_raw);
  PairTab<double>* tabd = reinterpret_cast<PairTab<double>*>(
      smem_raw + ((sizeof(PairTab<R>) * nrow + 15) / 16) * 16);
  {
    const int words = nrow * int(sizeof(PairTab<R>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(a.tab);
    int* dst = reinterpret_cast<int*>(tab);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  if constexpr (std::is_same<R, float>::value) {
    const int words = nrow * int(sizeof(PairTab<double>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(a.tabd);
    int* dst = reinterpret_cast<int*>(tabd);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  const bool ev = ev_mode == 1 || (ev_mode == 2 && a.st->ev);
  if (ev)
    pair_body<R, CG, true>(a.nslots, a.pos, a.nbr, a.cnt, a.perm, tab, tabd, a.nt, a.sx, a.sy, a.sz, a.sxd,
                           a.syd, a.szd, a.f_out, a.partial);
  else
    pair_body<R, CG, false>(a.nslots, a.pos, a.nbr, a.cnt, a.perm, tab, tabd, a.nt, a.sx, a.sy, a.sz, a.sxd,
                            a.syd, a.szd, a.f_out, a.partial);
}

template <typename R>
static cudaError_t launch_pairs_t(relres_ctx* c, int ev_mode, int which) {
  using F = typename std::conditional<std::is_same<R, float>::value, float4, double>::type;
  const double unit = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  const R sx = R(c->box[0] / unit), sy = R(c->box[1] / unit), sz = R(c->box[2] / unit);
  const double sxd = c->box[0] / 4294967296.0, syd = c->box[1] / 4294967296.0,
               szd = c->box[2] / 4294967296.0;
  const int nrow = c->n_types * c->n_types;
  size_t smem = ((sizeof(PairTab<R>) * nrow + 15) / 16) * 16;
  if (std::is_same<R, float>::value) smem += sizeof(PairTab<double>) * nrow;
  const typename PosOf<R>::T* pfg;
  const typename PosOf<R>::T* pcg;
  if constexpr (std::is_same<R, float>::value) {
    pfg = c->d_pos_fg;
    pcg = c->d_pos_cg;
  } else {
    pfg = c->d_pos_fg64;
    pcg = c->d_pos_cg64;
  }
  const PairTab<R>* tab = static_cast<const PairTab<R>*>(c->d_tab);
  const PairTab<double>* tabd = static_cast<const PairTab<double>*>(c->d_tabd);
  if (which & 1) {
    PairArgs<R> a{c->n, pfg, c->d_nbr_fg, c->d_cnt_fg, c->d_perm_fg, tab, tabd, c->n_types, sx, sy, sz,
                  sxd, syd, szd, static_cast<F*>(c->d_f_fg), c->d_part_fg, c->d_state};
    k_pair<R, false><<<(c->n + kThreads - 1) / kThreads, kThreads, smem, c->stream>>>(a, ev_mode);
    RELRES_LAUNCHED(c);
  }
  if ((which & 2) && c->has_cg && c->n_h > 0) {
    PairArgs<R> a{c->n_h, pcg, c->d_nbr_cg, c->d_cnt_cg, c->d_perm_cg, tab, tabd, c->n_types, sx, sy, sz,
                  sxd, syd, szd, static_cast<F*>(c->d_f_cg), c->d_part_cg, c->d_state};
    k_pair<R, true><<<(c->n_h + kThreads - 1) / kThreads, kThreads, smem, c->stream>>>(a, ev_mode);
    RELRES_LAUNCHED(c);
  }
  return cudaGetLastError();
}

cudaError_t launch_pairs(relres_ctx* c, int ev_mode, int which) {
  return c->fp64 ? launch_pairs_t<double>(c, ev_mode, which) : launch_pairs_t<float>(c, ev_mode, which);
}

}  // namespace relres
