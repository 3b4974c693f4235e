// RelRes pair kernel: Eq. 20 of the paper (Section 2.5) over the two lists.
//
// The potential is evaluated split exactly into an FG part (on the FG list:
// every atom, partners within r_s+) and a CG part (on the CG list: hybrid
// sites, partners within r_c+), see PairTab in relres_internal.h.  Forces
// never depend on a shift constant, so the split changes nothing but which
// list carries which term.  One launch covers both lists: the first blocks
// walk the CG list (fewer, longer-running slots, so they start first), the
// rest walk the FG list.
//
// One thread owns one sorted slot and walks its full list four entries at a
// time.  The list is stored in chunks of four (entry k of slot s at int
// (((k >> 2) * nslots + s) << 2) + (k & 3)), so a warp reads 512 contiguous
// bytes of indices per chunk with one 16-byte streaming load per thread, and
// the next chunk's indices are requested before the current chunk is
// evaluated.  The four partner positions (16-byte packed x, y, z, type, L1/L2
// resident thanks to the Morton cell order) are gathered together, then each
// entry gets an exact wrapped integer difference converted to FP32 and its
// region selected without branches.  The owner accumulates its force in
// registers and writes it once (no atomics).  Energy and virial are computed
// only on the steps that need them (EV template): they are reduced per block
// (warp shuffles, then shared memory) and added to 64-bit fixed-point
// accumulators with integer atomics.  The FP64 variant (R = double) reads 64-bit fixed-point
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

template <typename R>
using ForceOut = typename std::conditional<std::is_same<R, float>::value, float4, double>::type;

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

// FG part for one entry (FP64 path and FP64 energies).  Returns false outside r_s+.
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

// CG part for one entry (FP64 path and FP64 energies).  Returns false outside r_c+.
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

// FP32 force coefficients of one type pair, packed for 16-byte shared-memory
// loads (built in shared memory from PairTab<float> at kernel start).
struct FgRow {
  float4 a;  // r_s-^2, r_s+^2, 48 eps sig^12, 24 eps sig^6
  float4 b;  // r_s-, derivative of f_{s-}^{FG}: g1, 2 g2, 3 g3
  float4 c;  // 4 g4, -, -, -
};
struct CgRow {
  float4 a;  // r_s-^2, r_s+^2, r_c-^2, r_c+^2
  float4 b;  // r_s-, 3 gamma_3+, 4 gamma_4+, r_c-
  float4 c;  // 48 eps sig^12, 24 eps sig^6 (CG), derivative of f_{c-}^{CG}: g1, 2 g2
  float4 d;  // 3 g3, 4 g4, -, -
};

__device__ __forceinline__ void pack_rows(const PairTab<float>& t, FgRow& f, CgRow& g) {
  f.a = make_float4(t.rsm2, t.rsp2, t.f12f, t.f6f);
  f.b = make_float4(t.rsm, t.fgd[0], t.fgd[1], t.fgd[2]);
  f.c = make_float4(t.fgd[3], 0.f, 0.f, 0.f);
  g.a = make_float4(t.rsm2, t.rsp2, t.rcm2, t.rcp2);
  g.b = make_float4(t.rsm, t.ond3, t.ond4, t.rcm);
  g.c = make_float4(t.f12c, t.f6c, t.cgod[0], t.cgod[1]);
  g.d = make_float4(t.cgod[2], t.cgod[3], 0.f, 0.f);
}

// -dU/dr / r of the FG part, every region evaluated and the right one
// selected (same arithmetic as fg_term<float>).  r2 >= r_s+^2 gives 0.
__device__ __forceinline__ float fg_force(const FgRow& T, float r2) {
  const float4 a = T.a, b = T.b;
  const float g4 = T.c.x;
  const float r2i = __frcp_rn(r2);
  const float r6i = r2i * r2i * r2i;
  const float flj = r6i * (a.z * r6i - a.w) * r2i;
  const float ri = rsqrtf(r2);
  const float d = r2 * ri - b.x;
  const float fp = ((g4 * d + b.w) * d + b.z) * d + b.y;
  const float fsh = -fp * ri;
  const float fr = r2 < a.x ? flj : fsh;
  return r2 < a.y ? fr : 0.f;
}

// -dU/dr / r of the CG part (same arithmetic as cg_term<float>): zero below
// r_s- (the constant region) and from r_c+ on.
__device__ __forceinline__ float cg_force(const CgRow& T, float r2) {
  const float4 a = T.a, b = T.b, c = T.c;
  const float2 dd = make_float2(T.d.x, T.d.y);
  const float ri = rsqrtf(r2);
  const float r = r2 * ri;
  const float d = r - b.x;
  const float fon = -(d * d * (b.z * d + b.y)) * ri;
  const float r2i = ri * ri;
  const float r6i = r2i * r2i * r2i;
  const float flj = r6i * (c.x * r6i - c.y) * r2i;
  const float e = r - b.w;
  const float foff = -(((dd.y * e + dd.x) * e + c.w) * e + c.z) * ri;
  float fr = r2 < a.z ? flj : foff;
  fr = r2 < a.y ? fon : fr;
  return (r2 < a.x || !(r2 < a.w)) ? 0.f : fr;
}

__device__ __forceinline__ double dfix32d(int a, int b, double scale) {
  return double(int(unsigned(a) - unsigned(b))) * scale;
}

template <typename R>
struct ListWalk {
  int nslots;
  const typename PosOf<R>::T* pos;
  const int* nbr;
  const int* cnt;
  const int* perm;
  ForceOut<R>* f_out;
  long long* acc;  // kNQ accumulators of this list (energy, six virial components)
};

template <typename R>
struct PairLaunch {
  int nblk_cg;  // blocks [0, nblk_cg) walk the CG list, the rest the FG list
  ListWalk<R> fg, cg;
  const PairTab<R>* tab;
  const PairTab<double>* tabd;  // FP64 table: energies of the FP32 path are evaluated in FP64
  int nt;
  R sx, sy, sz;
  double sxd, syd, szd;  // L / 2^32 (FP32 path) for the FP64 energy
};

struct SmemTabs {
  const void* tab;
  const PairTab<double>* tabd;
  const FgRow* fgr;
  const CgRow* cgr;
};

// Per-thread accumulators of one walk.
template <typename R>
struct Acc {
  R fx = R(0), fy = R(0), fz = R(0);
  R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  double e = 0.0;
};

template <typename R, bool CG, bool EV>
__device__ __forceinline__ void entry(const typename PosOf<R>::T& pi, const typename PosOf<R>::T& pj,
                                      bool valid, int row0, const SmemTabs& S, const PairLaunch<R>& a,
                                      Acc<R>& A) {
  R dx, dy, dz;
  delta(pi, pj, a.sx, a.sy, a.sz, dx, dy, dz);
  const int row = row0 + ptype(pj);
  if constexpr (std::is_same<R, float>::value) {
    float r2 = dx * dx + dy * dy + dz * dz;
    r2 = valid ? r2 : 3.0e38f;  // padding entry: past every cutoff
    const float fr = CG ? cg_force(S.cgr[row], r2) : fg_force(S.fgr[row], r2);
    A.fx += fr * dx;
    A.fy += fr * dy;
    A.fz += fr * dz;
    if (EV) {
      A.w[0] += fr * dx * dx;
      A.w[1] += fr * dy * dy;
      A.w[2] += fr * dz * dz;
      A.w[3] += fr * dx * dy;
      A.w[4] += fr * dx * dz;
      A.w[5] += fr * dy * dz;
      if (valid) {
        const double ex = dfix32d(pi.x, pj.x, a.sxd), ey = dfix32d(pi.y, pj.y, a.syd),
                     ez = dfix32d(pi.z, pj.z, a.szd);
        const PairTab<double>& Td = S.tabd[row];
        double frd, epd;
        if (CG ? cg_term<double, true>(Td, ex * ex + ey * ey + ez * ez, frd, epd)
               : fg_term<double, true>(Td, ex * ex + ey * ey + ez * ez, frd, epd))
          A.e += epd;
      }
    }
  } else {
    if (!valid) return;
    const R r2 = dx * dx + dy * dy + dz * dz;
    const PairTab<R>& T = static_cast<const PairTab<R>*>(S.tab)[row];
    R fr, ep;
    const bool hit = CG ? cg_term<R, EV>(T, r2, fr, ep) : fg_term<R, EV>(T, r2, fr, ep);
    if (hit) {
      A.fx += fr * dx;
      A.fy += fr * dy;
      A.fz += fr * dz;
      if (EV) {
        A.e += ep;
        A.w[0] += fr * dx * dx;
        A.w[1] += fr * dy * dy;
        A.w[2] += fr * dz * dz;
        A.w[3] += fr * dx * dy;
        A.w[4] += fr * dx * dz;
        A.w[5] += fr * dy * dz;
      }
    }
  }
}

// One slot's walk over its list, four entries per iteration.
template <typename R, bool CG, bool EV>
__device__ __forceinline__ void walk(const ListWalk<R>& L, int blk, const SmemTabs& S,
                                     const PairLaunch<R>& a) {
  const int s = blk * blockDim.x + threadIdx.x;
  Acc<R> A;
  if (s < L.nslots) {
    const auto pi = L.pos[s];
    const int row0 = ptype(pi) * a.nt;
    const int m = L.cnt[s];
    const int nch = (m + 3) >> 2;
    const int4* nb4 = reinterpret_cast<const int4*>(L.nbr) + s;
    int4 jj = make_int4(s, s, s, s);
    if (nch > 0) jj = __ldcs(nb4);
    for (int ch = 0; ch < nch; ++ch) {
      int4 jn = jj;
      if (ch + 1 < nch) jn = __ldcs(nb4 + size_t(ch + 1) * L.nslots);
      const int rem = m - 4 * ch;  // >= 1
      const int j1 = rem > 1 ? jj.y : s, j2 = rem > 2 ? jj.z : s, j3 = rem > 3 ? jj.w : s;
      const auto p0 = load_pos(L.pos, jj.x);
      const auto p1 = load_pos(L.pos, j1);
      const auto p2 = load_pos(L.pos, j2);
      const auto p3 = load_pos(L.pos, j3);
      entry<R, CG, EV>(pi, p0, true, row0, S, a, A);
      entry<R, CG, EV>(pi, p1, rem > 1, row0, S, a, A);
      entry<R, CG, EV>(pi, p2, rem > 2, row0, S, a, A);
      entry<R, CG, EV>(pi, p3, rem > 3, row0, S, a, A);
      jj = jn;
    }
    store_force(L.f_out, L.perm[s], A.fx, A.fy, A.fz);
  }
  if (EV) {
    // per-thread sums are R (FP64 for the energy); the block sum is taken in FP64
    double accd[kNQ];
    accd[0] = A.e;
#pragma unroll
    for (int q = 0; q < 6; ++q) accd[q + 1] = double(A.w[q]);
    __shared__ double sh[(kThreads / 32) * kNQ];
    block_sum<double, kNQ>(accd, sh);
    if (threadIdx.x == 0) {
      // full lists: every pair was visited from both ends
#pragma unroll
      for (int q = 0; q < kNQ; ++q) acc_add(L.acc + q, 0.5 * accd[q]);
    }
  }
}

template <typename R, bool EV>
__global__ void __launch_bounds__(kThreads) k_pair(PairLaunch<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = a.nt * a.nt;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = smem_raw + off;
    off += (bytes + 15) / 16 * 16;
    return p;
  };
  SmemTabs S{};
  if constexpr (std::is_same<R, float>::value) {
    FgRow* fgr = reinterpret_cast<FgRow*>(carve(sizeof(FgRow) * nrow));
    CgRow* cgr = reinterpret_cast<CgRow*>(carve(sizeof(CgRow) * nrow));
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) pack_rows(a.tab[r], fgr[r], cgr[r]);
    S.fgr = fgr;
    S.cgr = cgr;
    if (EV) {
      PairTab<double>* tabd = reinterpret_cast<PairTab<double>*>(carve(sizeof(PairTab<double>) * nrow));
      const int words = nrow * int(sizeof(PairTab<double>) / sizeof(int));
      const int* src = reinterpret_cast<const int*>(a.tabd);
      int* dst = reinterpret_cast<int*>(tabd);
      for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
      S.tabd = tabd;
    }
  } else {
    PairTab<R>* tab = reinterpret_cast<PairTab<R>*>(carve(sizeof(PairTab<R>) * nrow));
    const int words = nrow * int(sizeof(PairTab<R>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(a.tab);
    int* dst = reinterpret_cast<int*>(tab);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    S.tab = tab;
  }
  __syncthreads();
  if (int(blockIdx.x) < a.nblk_cg)
    walk<R, true, EV>(a.cg, blockIdx.x, S, a);
  else
    walk<R, false, EV>(a.fg, blockIdx.x - a.nblk_cg, S, a);
}

template <typename R>
static size_t pair_smem(int nt, bool ev) {
  const size_t nrow = size_t(nt) * nt;
  auto up = [](size_t b) { return (b + 15) / 16 * 16; };
  if (std::is_same<R, float>::value)
    return up(sizeof(FgRow) * nrow) + up(sizeof(CgRow) * nrow) + (ev ? up(sizeof(PairTab<double>) * nrow) : 0);
  return up(sizeof(PairTab<R>) * nrow);
}

template <typename R>
static cudaError_t launch_pairs_t(relres_ctx* c, bool ev, int which) {
  const double unit = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  PairLaunch<R> a{};
  a.sx = R(c->box[0] / unit);
  a.sy = R(c->box[1] / unit);
  a.sz = R(c->box[2] / unit);
  a.sxd = c->box[0] / 4294967296.0;
  a.syd = c->box[1] / 4294967296.0;
  a.szd = c->box[2] / 4294967296.0;
  a.nt = c->n_types;
  a.tab = static_cast<const PairTab<R>*>(c->d_tab);
  a.tabd = static_cast<const PairTab<double>*>(c->d_tabd);
  const typename PosOf<R>::T* pfg;
  const typename PosOf<R>::T* pcg;
  if constexpr (std::is_same<R, float>::value) {
    pfg = c->d_pos_fg;
    pcg = c->d_pos_cg;
  } else {
    pfg = c->d_pos_fg64;
    pcg = c->d_pos_cg64;
  }
  const bool do_fg = (which & 1) != 0;
  const bool do_cg = (which & 2) && c->has_cg && c->n_h > 0;
  const int nb_fg = do_fg ? (c->n + kThreads - 1) / kThreads : 0;
  const int nb_cg = do_cg ? (c->n_h + kThreads - 1) / kThreads : 0;
  if (nb_fg + nb_cg == 0) return cudaSuccess;
  a.nblk_cg = nb_cg;
  a.fg = ListWalk<R>{c->n, pfg, c->d_nbr_fg, c->d_cnt_fg, c->d_perm_fg,
                     static_cast<ForceOut<R>*>(c->d_f_fg), c->d_acc + kAccFg};
  // without a CG list the CG walk is never entered; its pointers are stand-ins
  a.cg = do_cg ? ListWalk<R>{c->n_h, pcg, c->d_nbr_cg, c->d_cnt_cg, c->d_perm_cg,
                             static_cast<ForceOut<R>*>(c->d_f_cg), c->d_acc + kAccCg}
               : a.fg;
  const size_t smem = pair_smem<R>(c->n_types, ev);
  if (ev)
    k_pair<R, true><<<nb_cg + nb_fg, kThreads, smem, c->stream>>>(a);
  else
    k_pair<R, false><<<nb_cg + nb_fg, kThreads, smem, c->stream>>>(a);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_pairs(relres_ctx* c, bool ev, int which) {
  return c->fp64 ? launch_pairs_t<double>(c, ev, which) : launch_pairs_t<float>(c, ev, which);
}

}  // namespace relres
