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
// only on the steps that need them (EV template); pair energies of the FP32
// path are float-float (see FgE), reduced per block in FP64 (warp shuffles,
// then shared memory) and added to 64-bit fixed-point accumulators with
// integer atomics.  The FP64 variant (R = double) reads 64-bit fixed-point
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

__device__ __forceinline__ float recip(float x) { return rcp_nr(x); }
__device__ __forceinline__ double recip(double x) { return rcp_d(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt_d(x); }

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
  float4 a;  // 4 g4, r_s+^2, 48 eps sig^12, 24 eps sig^6
  float4 b;  // r_s-, derivative of f_{s-}^{FG}: g1, 2 g2, 3 g3
};
struct CgRow {
  float4 a;  // r_s+^2, r_c+^2, r_s-, r_c-
  float4 b;  // 3 gamma_3+, 4 gamma_4+, 48 eps sig^12, 24 eps sig^6 (CG)
  float4 c;  // derivative of f_{c-}^{CG}: g1, 2 g2, 3 g3, 4 g4
};

// Energy constants of one type pair for the FP32 path (energy steps) as
// float-float values.  Pair energies of energy steps are evaluated in
// float-float arithmetic (~48-bit): in FP32 alone, rounding that is the same
// for every pair of a type (constants, the box scale, approximate
// reciprocals) biases the total, and the FG and CG parts largely cancel in
// it, so 1e-7 of the total is out of reach; FP64 proper runs at a small
// fraction of the FP32 rate on this part.
struct FgE {
  ff c12, c6, shift, rsm, g[5];
};
struct CgE {
  ff c12, c6, gam, rsm, rcm, on0, on3, on4, close, g[5];
};
__device__ __forceinline__ ff split_ff(double v) {
  const float h = float(v);
  return ff{h, float(v - double(h))};
}
__device__ __forceinline__ void pack_energy_rows(const PairTab<double>& t, FgE& f, CgE& c) {
  f.c12 = split_ff(t.c12f);
  f.c6 = split_ff(t.c6f);
  f.shift = split_ff(t.e_fg_shift);
  f.rsm = split_ff(t.rsm);
  c.c12 = split_ff(t.c12c);
  c.c6 = split_ff(t.c6c);
  c.gam = split_ff(t.gam_cm);
  c.rsm = split_ff(t.rsm);
  c.rcm = split_ff(t.rcm);
  c.on0 = split_ff(t.on0);
  c.on3 = split_ff(t.on3);
  c.on4 = split_ff(t.on4);
  c.close = split_ff(t.e_cg_close);
  for (int m = 0; m < 5; ++m) {
    f.g[m] = split_ff(t.fg[m]);
    c.g[m] = split_ff(t.cgo[m]);
  }
}
__device__ __forceinline__ ff poly5_ff(const ff (&g)[5], ff d) {
  ff p = g[4];
#pragma unroll
  for (int m = 3; m >= 0; --m) p = ff_add(ff_mul(p, d), g[m]);
  return p;
}
__device__ __forceinline__ ff lj_ff(const ff& c12, const ff& c6, ff r2i) {
  const ff r6i = ff_mul(ff_mul(r2i, r2i), r2i);
  return ff_sub(ff_mul(c12, ff_mul(r6i, r6i)), ff_mul(c6, r6i));
}
// FG energy of a pair inside r_s+ (regions chosen on the leading part: the
// potential is C2 at r_s-, so a pair rounded across it changes nothing)
__device__ __forceinline__ ff fg_energy_ff(const FgE& T, float rsm2, ff r2) {
  const ff e = r2.hi < rsm2 ? lj_ff(T.c12, T.c6, ff_rcp(r2)) : poly5_ff(T.g, ff_sub(ff_sqrt(r2), T.rsm));
  return ff_sub(e, T.shift);
}
// CG energy of a pair inside r_c+
__device__ __forceinline__ ff cg_energy_ff(const CgE& T, float4 radii2, ff r2) {
  if (r2.hi < radii2.x) return T.close;
  ff e;
  if (r2.hi < radii2.y) {
    const ff d = ff_sub(ff_sqrt(r2), T.rsm);
    const ff d3 = ff_mul(ff_mul(d, d), d);
    e = ff_add(T.on0, ff_mul(d3, ff_add(ff_mul(T.on4, d), T.on3)));
  } else if (r2.hi < radii2.z) {
    e = lj_ff(T.c12, T.c6, ff_rcp(r2));
  } else {
    e = poly5_ff(T.g, ff_sub(ff_sqrt(r2), T.rcm));
  }
  return ff_sub(e, T.gam);
}

__device__ __forceinline__ void pack_rows(const PairTab<float>& t, FgRow& f, CgRow& g) {
  f.a = make_float4(t.fgd[3], t.rsp2, t.f12f, t.f6f);
  f.b = make_float4(t.rsm, t.fgd[0], t.fgd[1], t.fgd[2]);
  g.a = make_float4(t.rsp2, t.rcp2, t.rsm, t.rcm);
  g.b = make_float4(t.ond3, t.ond4, t.f12c, t.f6c);
  g.c = make_float4(t.cgod[0], t.cgod[1], t.cgod[2], t.cgod[3]);
}

// -dU/dr / r of the FG part, every region evaluated and the right one
// selected (the arithmetic of fg_term, the LJ core chosen by the sign of
// r - r_s-).  r2 >= r_s+^2 gives 0.
__device__ __forceinline__ float fg_force(const FgRow& T, float r2) {
  const float4 a = T.a, b = T.b;
  const float g4 = a.x;
  const float r2i = rcp_nr(r2);
  const float r6i = r2i * r2i * r2i;
  const float flj = r6i * (a.z * r6i - a.w) * r2i;
  const float ri = rsqrtf(r2);
  const float d = r2 * ri - b.x;
  const float fp = ((g4 * d + b.w) * d + b.z) * d + b.y;
  const float fsh = -fp * ri;
  const float fr = d < 0.f ? flj : fsh;  // r < r_s-: LJ core
  return r2 < a.y ? fr : 0.f;
}

// -dU/dr / r of the CG part (the arithmetic of cg_term, the regions below
// r_s- and r_c- chosen by the signs of r - r_s- and r - r_c-): zero below
// r_s- (the constant region) and from r_c+ on.
__device__ __forceinline__ float cg_force(const CgRow& T, float r2) {
  const float4 a = T.a, b = T.b, c = T.c;
  const float ri = rsqrtf(r2);
  const float r = r2 * ri;
  const float d = r - a.z;
  const float fon = -(d * d * (b.y * d + b.x)) * ri;
  const float r2i = ri * ri;
  const float r6i = r2i * r2i * r2i;
  const float flj = r6i * (b.z * r6i - b.w) * r2i;
  const float e = r - a.w;
  const float foff = -(((c.w * e + c.z) * e + c.y) * e + c.x) * ri;
  float fr = e < 0.f ? flj : foff;
  fr = r2 < a.x ? fon : fr;
  return (d < 0.f || !(r2 < a.y)) ? 0.f : fr;
}

// (r_s-^2, r_s+^2, r_c-^2, r_c+^2) of a CG row, for the energy regions
__device__ __forceinline__ float4 cg_radii2(const CgRow& T) {
  return make_float4(T.a.z * T.a.z, T.a.x, T.a.w * T.a.w, T.a.y);
}


template <typename R>
struct ListWalk {
  int nslots;
  const typename PosOf<R>::T* pos;
  const int* nbr;  // the list walked (pruned when pruning is on)
  const int* cnt;
  const int* perm;
  ForceOut<R>* f_out;
  long long* acc;  // kNQ accumulators of this list (energy, six virial components)
  // pruning launches (PRN): walk the full list and write the pruned one
  const int* nbr_full;
  const int* cnt_full;
  int* nbr_in;
  int* cnt_in;
  R rp2;  // (interaction cutoff + delta + slack)^2
  unsigned long long* tot_in;
};

template <typename R>
struct PairLaunch {
  int nblk_cg;  // blocks [0, nblk_cg) walk the CG list, the rest the FG list
  ListWalk<R> fg, cg;
  const PairTab<R>* tab;
  const PairTab<double>* tabd;  // FP64 table: source of the split energy constants of the FP32 path
  int nt;
  R sx, sy, sz;
  float sxl, syl, szl;  // FP32 path: lo parts of L / 2^32 (float-float energies)
  const unsigned* gate;  // device flag word of the step
  int prune_on;          // prune on this launch if F_REBUILD or F_PRUNE is set (TPA = 1 only)
  int4* ref_p;  // PRN: positions of this pruning pass, caller order (FG walk)
  DevState* st;
};

struct SmemTabs {
  const void* tab;
  const FgRow* fgr;
  const CgRow* cgr;
  const FgE* fge;
  const CgE* cge;
  int4* evq;  // FP32 energy steps: kEvQueue queued pairs per warp
};

// Per-thread accumulators of one walk.  The owner's force sum of the FP32
// path is kept in one of three ways (ACC, relres_set_force_accumulation):
// FP32 running sums (fx, fy, fz); compensated sums, where the (up to) four
// entries of a list chunk are summed in FP32 (kx, ...) and each chunk sum is
// added to a float-float total (fx + cx, ...) with an error-free two-sum; or
// FP64 running sums (dfx, ...), one conversion and FP64 add per entry.  The
// members a variant does not use are removed by the compiler.
template <typename R>
struct Acc {
  R fx = R(0), fy = R(0), fz = R(0);
  float kx = 0.f, ky = 0.f, kz = 0.f;
  float cx = 0.f, cy = 0.f, cz = 0.f;
  double dfx = 0.0, dfy = 0.0, dfz = 0.0;
  R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  R e = R(0);            // FP64 path: per-thread energy
  ff eff = ff{0.f, 0.f};  // FP32 path: per-thread energy in float-float
};

template <int ACC>
__device__ __forceinline__ void acc_force(Acc<float>& A, float tx, float ty, float tz) {
  if constexpr (ACC == RELRES_ACC_COMPENSATED) {
    A.kx += tx;
    A.ky += ty;
    A.kz += tz;
  } else if constexpr (ACC == RELRES_ACC_FP64) {
    A.dfx += double(tx);
    A.dfy += double(ty);
    A.dfz += double(tz);
  } else {
    A.fx += tx;
    A.fy += ty;
    A.fz += tz;
  }
}

// end of a list chunk: the compensated variant moves the chunk sum into its
// float-float total
template <int ACC>
__device__ __forceinline__ void acc_chunk(Acc<float>& A) {
  if constexpr (ACC == RELRES_ACC_COMPENSATED) {
    const ff sx = ff_two_sum(A.fx, A.kx), sy = ff_two_sum(A.fy, A.ky), sz = ff_two_sum(A.fz, A.kz);
    A.fx = sx.hi;
    A.fy = sy.hi;
    A.fz = sz.hi;
    A.cx = __fadd_rn(A.cx, sx.lo);
    A.cy = __fadd_rn(A.cy, sy.lo);
    A.cz = __fadd_rn(A.cz, sz.lo);
    A.kx = A.ky = A.kz = 0.f;
  }
}
template <int ACC>
__device__ __forceinline__ void acc_chunk(Acc<double>&) {}

// the owner's force sum rounded to FP32 (the width of the force buffers)
template <int ACC>
__device__ __forceinline__ void acc_final(Acc<float>& A) {
  if constexpr (ACC == RELRES_ACC_COMPENSATED) {
    A.fx = __fadd_rn(A.fx, A.cx);
    A.fy = __fadd_rn(A.fy, A.cy);
    A.fz = __fadd_rn(A.fz, A.cz);
  } else if constexpr (ACC == RELRES_ACC_FP64) {
    A.fx = float(A.dfx);
    A.fy = float(A.dfy);
    A.fz = float(A.dfz);
  }
}
template <int ACC>
__device__ __forceinline__ void acc_final(Acc<double>&) {}

// One list entry; returns its squared distance (past every cutoff for a
// padding entry), which a pruning launch compares with the pruning radius.
template <typename R, bool CG, bool EV, int ACC, bool EN = EV>
__device__ __forceinline__ R entry(const typename PosOf<R>::T& pi, const typename PosOf<R>::T& pj,
                                   bool valid, int row0, const SmemTabs& S, const PairLaunch<R>& a,
                                   Acc<R>& A) {
  R dx, dy, dz;
  delta(pi, pj, a.sx, a.sy, a.sz, dx, dy, dz);
  const int row = row0 + ptype(pj);
  if constexpr (std::is_same<R, float>::value) {
    float r2 = dx * dx + dy * dy + dz * dz;
    r2 = valid ? r2 : 3.0e38f;  // padding entry: past every cutoff
    const float fr = CG ? cg_force(S.cgr[row], r2) : fg_force(S.fgr[row], r2);
    acc_force<ACC>(A, fr * dx, fr * dy, fr * dz);
    if (EV) {
      A.w[0] += fr * dx * dx;
      A.w[1] += fr * dy * dy;
      A.w[2] += fr * dz * dz;
      A.w[3] += fr * dx * dy;
      A.w[4] += fr * dx * dz;
      A.w[5] += fr * dy * dz;
      // float-float energy inside the cutoff only (padding entries carry
      // r2 = 3e38; the energy and its slope vanish at the cutoff, so the FP32
      // decision is harmless), from the exact integer coordinate differences
      const float rcut2 = CG ? S.cgr[row].a.y : S.fgr[row].a.y;
      if (EN && r2 < rcut2) {
        const ff ex = ff_fixed_diff32(pi.x, pj.x, ff{a.sx, a.sxl});
        const ff ey = ff_fixed_diff32(pi.y, pj.y, ff{a.sy, a.syl});
        const ff ez = ff_fixed_diff32(pi.z, pj.z, ff{a.sz, a.szl});
        const ff r2e = ff_add(ff_add(ff_mul(ex, ex), ff_mul(ey, ey)), ff_mul(ez, ez));
        A.eff = ff_add(A.eff, CG ? cg_energy_ff(S.cge[row], cg_radii2(S.cgr[row]), r2e)
                                 : fg_energy_ff(S.fge[row], S.fgr[row].b.x * S.fgr[row].b.x, r2e));
      }
    }
    return r2;
  } else {
    if (!valid) return R(1e300);
    const R r2 = dx * dx + dy * dy + dz * dz;
    const PairTab<R>& T = static_cast<const PairTab<R>*>(S.tab)[row];
    R fr, ep;
    const bool hit = CG ? cg_term<R, EV>(T, r2, fr, ep) : fg_term<R, EV>(T, r2, fr, ep);
    if (hit) {
      // one rounding per term (fma): the operation the ordered several-lane
      // walk repeats (walk_ordered), so both give the same bits
      A.fx = fma(fr, dx, A.fx);
      A.fy = fma(fr, dy, A.fy);
      A.fz = fma(fr, dz, A.fz);
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
    return r2;
  }
}

// Float-float energy of one pair from its exact 32-bit coordinate
// differences d = (pi - pj).xyz and type-pair row d.w (the arithmetic of the
// energy part of entry()).
// (one copy per list kind, called from the queue drains: inlined at each of
// them the float-float code overflowed the instruction cache)
template <bool CG>
__device__ __noinline__ ff pair_energy_ff(int4 d, const SmemTabs& S, const PairLaunch<float>& a) {
  const ff ex = ff_fixed_diff32(d.x, 0, ff{a.sx, a.sxl});
  const ff ey = ff_fixed_diff32(d.y, 0, ff{a.sy, a.syl});
  const ff ez = ff_fixed_diff32(d.z, 0, ff{a.sz, a.szl});
  const ff r2e = ff_add(ff_add(ff_mul(ex, ex), ff_mul(ey, ey)), ff_mul(ez, ez));
  const int row = d.w;
  return CG ? cg_energy_ff(S.cge[row], cg_radii2(S.cgr[row]), r2e)
            : fg_energy_ff(S.fge[row], S.fgr[row].b.x * S.fgr[row].b.x, r2e);
}

// Energy steps of the FP32 path: each pair's energy is evaluated once (by the
// owner of the lower slot; the lists hold every pair from both ends) and not
// where it is met: the warp queues (pair, row) items in shared memory and
// evaluates 32 of them at a time, one per lane, so no lane idles through the
// float-float arithmetic of another's entry.  kEvQueue items per warp: fewer
// than 32 wait between two drains, and one pass adds at most 32.
constexpr int kEvQueue = 64;
struct EvQueue {
  int4* q;  // this warp's kEvQueue items
  int n;    // items waiting (the same in every lane)
};

template <bool CG>
__device__ __forceinline__ void ev_push(EvQueue& Q, bool need, int4 item, const SmemTabs& S,
                                        const PairLaunch<float>& a, ff& eff) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(0xffffffffu, need);
  if (need) Q.q[Q.n + __popc(b & ((1u << lane) - 1u))] = item;
  Q.n += __popc(b);
  if (Q.n >= 32) {
    __syncwarp();
    const int4 d = Q.q[Q.n - 32 + lane];
    __syncwarp();
    Q.n -= 32;
    eff = ff_add(eff, pair_energy_ff<CG>(d, S, a));
  }
}

__device__ __forceinline__ int4 fixed_delta(const int4& pi, const int4& pj, int row) {
  return make_int4(int(unsigned(pi.x) - unsigned(pj.x)), int(unsigned(pi.y) - unsigned(pj.y)),
                   int(unsigned(pi.z) - unsigned(pj.z)), row);
}

__device__ __forceinline__ int4 ref_of(const int4& p) { return p; }
__device__ __forceinline__ int4 ref_of(const Pos64& p) {
  return make_int4(int(p.x >> 32), int(p.y >> 32), int(p.z >> 32), int(p.t));
}

// FP64 force factor of one entry and its coordinate difference (the
// arithmetic of entry()); zero for a padding entry or a pair past the cutoff.
template <bool CG>
__device__ __forceinline__ double term64(const Pos64& pi, const Pos64& pj, bool valid, int row0, const SmemTabs& S,
                                         const PairLaunch<double>& a, double d[3]) {
  double dx, dy, dz;
  delta(pi, pj, a.sx, a.sy, a.sz, dx, dy, dz);
  const double r2 = dx * dx + dy * dy + dz * dz;
  const PairTab<double>& T = static_cast<const PairTab<double>*>(S.tab)[row0 + ptype(pj)];
  double fr = 0.0, ep;
  const bool hit = valid && (CG ? cg_term<double, false>(T, r2, fr, ep) : fg_term<double, false>(T, r2, fr, ep));
  d[0] = hit ? dx : 0.0;
  d[1] = hit ? dy : 0.0;
  d[2] = hit ? dz : 0.0;
  return hit ? fr : 0.0;
}

// FP64 forces of small systems (too few slots to occupy the part with one
// thread each): TPA lanes per slot, and the same bits as one lane.  In each
// round the TPA lanes of a slot evaluate one chunk each (TPA x 4 consecutive
// entries); lanes 0, 1 and 2 of the slot then add the x, y and z terms of
// those entries in list order with the one-lane walk's operation (fma),
// taking each entry's force factor and difference from the lane that
// evaluated it.  A padding entry or a pair past the cutoff adds fma(0, 0, f)
// = f.  Every lane of the warp runs the warp's largest number of rounds (the
// shuffles take all 32 lanes).
template <bool CG, int TPA>
__device__ __forceinline__ void walk_ordered(const ListWalk<double>& L, int blk, const SmemTabs& S,
                                             const PairLaunch<double>& a) {
  static_assert(TPA >= 4 && 32 % TPA == 0, "three lanes per slot add the components");
  const int t = blk * blockDim.x + threadIdx.x;
  const int s = t / TPA, q = t % TPA;
  const int base = (threadIdx.x & 31) - q;  // the slot's first lane in the warp
  const bool own = s < L.nslots;
  const int ss = own ? s : 0;  // a valid slot for the loads of the other lanes
  const Pos64 pi = L.pos[ss];
  const int row0 = ptype(pi) * a.nt;
  const int m = own ? L.cnt[s] : 0;
  const int nch = (m + 3) >> 2;
  const int nround_w = __reduce_max_sync(0xffffffffu, (nch + TPA - 1) / TPA);
  const int4* nb4 = reinterpret_cast<const int4*>(L.nbr) + ss;
  double f = 0.0;  // lanes 0, 1, 2 of the slot: its force component q
  for (int r = 0; r < nround_w; ++r) {
    const int ch = r * TPA + q;
    const int rem = ch < nch ? m - 4 * ch : 0;
    int4 jj = make_int4(ss, ss, ss, ss);
    if (rem > 0) jj = __ldcs(nb4 + size_t(ch) * L.nslots);
    const int jv[4] = {rem > 0 ? jj.x : ss, rem > 1 ? jj.y : ss, rem > 2 ? jj.z : ss, rem > 3 ? jj.w : ss};
    double fr[4], d[4][3];
#pragma unroll
    for (int e = 0; e < 4; ++e) fr[e] = term64<CG>(pi, load_pos(L.pos, jv[e]), rem > e, row0, S, a, d[e]);
    for (int k = 0; k < TPA; ++k) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const double frk = __shfl_sync(0xffffffffu, fr[e], base + k);
        const double xk = __shfl_sync(0xffffffffu, d[e][0], base + k);
        const double yk = __shfl_sync(0xffffffffu, d[e][1], base + k);
        const double zk = __shfl_sync(0xffffffffu, d[e][2], base + k);
        f = fma(frk, q == 0 ? xk : (q == 1 ? yk : zk), f);
      }
    }
  }
  if (own && q < 3) L.f_out[3 * size_t(L.perm[s]) + q] = f;
}

// One slot's walk over its list, four entries per iteration.  TPA lanes share
// one slot (threads per atom, chosen by the autotuner): lane q of the slot
// takes chunks q, q + TPA, ... and the partial forces are summed with warp
// shuffles.  Energy steps use TPA = 1.
// PRN (pruning launches, TPA = 1): the slot walks its full list, and every
// entry within the pruning radius is appended, in list order, to its pruned
// list; the forces are the same bits as a walk of the pruned list (a dropped
// entry adds exactly zero).
template <typename R, bool CG, bool EV, int TPA, bool PRN, int ACC>
__device__ __forceinline__ void walk(const ListWalk<R>& L, int blk, const SmemTabs& S,
                                     const PairLaunch<R>& a, bool first_block) {
  static_assert(!PRN || TPA == 1, "pruning launches use one thread per slot");
  const int t = blk * blockDim.x + threadIdx.x;
  const int s = t / TPA;
  const int q = t % TPA;
  Acc<R> A;
  int kept = 0;
  constexpr bool EVQ = EV && std::is_same<R, float>::value;  // queued energies (TPA = 1)
  static_assert(!EVQ || TPA == 1, "energy steps use one thread per slot");
  if constexpr (EVQ) {
    // every lane of the warp runs the same number of chunk passes (the
    // warp's longest list; lanes past their own list or past the last slot
    // add nothing) so that the queue's ballots see all 32 lanes
    EvQueue Q{S.evq + (threadIdx.x >> 5) * kEvQueue, 0};
    const bool own = s < L.nslots;
    const int ss = own ? s : 0;  // a valid slot for the loads of the other lanes
    const auto pi = L.pos[ss];
    const int row0 = ptype(pi) * a.nt;
    const int m = own ? (PRN ? L.cnt_full[s] : L.cnt[s]) : 0;
    const int nch = (m + 3) >> 2;
    const int nch_w = __reduce_max_sync(0xffffffffu, nch);
    const int4* nb4 = reinterpret_cast<const int4*>(PRN ? L.nbr_full : L.nbr) + ss;
    int4* out4 = reinterpret_cast<int4*>(L.nbr_in) + ss;
    int4 buf = make_int4(ss, ss, ss, ss);
    int4 jj = make_int4(ss, ss, ss, ss);
    if (nch > 0) jj = __ldcs(nb4);
    for (int ch = 0; ch < nch_w; ++ch) {
      const bool live = ch < nch;
      int4 jn = jj;
      if (ch + 1 < nch) jn = __ldcs(nb4 + size_t(ch + 1) * L.nslots);
      const int rem = live ? m - 4 * ch : 0;
      const int j0 = rem > 0 ? jj.x : ss, j1 = rem > 1 ? jj.y : ss, j2 = rem > 2 ? jj.z : ss,
                j3 = rem > 3 ? jj.w : ss;
      const auto p0 = load_pos(L.pos, j0);
      const auto p1 = load_pos(L.pos, j1);
      const auto p2 = load_pos(L.pos, j2);
      const auto p3 = load_pos(L.pos, j3);
      const R r0 = entry<R, CG, EV, ACC, false>(pi, p0, rem > 0, row0, S, a, A);
      const R r1 = entry<R, CG, EV, ACC, false>(pi, p1, rem > 1, row0, S, a, A);
      const R r2 = entry<R, CG, EV, ACC, false>(pi, p2, rem > 2, row0, S, a, A);
      const R r3 = entry<R, CG, EV, ACC, false>(pi, p3, rem > 3, row0, S, a, A);
      if (live) acc_chunk<ACC>(A);
      if (PRN && live) {
        keep_entry(r0 < L.rp2, j0, kept, buf, out4, L.nslots);
        keep_entry(r1 < L.rp2, j1, kept, buf, out4, L.nslots);
        keep_entry(r2 < L.rp2, j2, kept, buf, out4, L.nslots);
        keep_entry(r3 < L.rp2, j3, kept, buf, out4, L.nslots);
      }
      // energies of the pairs inside the cutoff, each from its lower slot
      const R rr[4] = {r0, r1, r2, r3};
      const int jv[4] = {j0, j1, j2, j3};
      const int4 pv[4] = {p0, p1, p2, p3};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = row0 + ptype(pv[e]);
        const float rcut2 = CG ? S.cgr[row].a.y : S.fgr[row].a.y;
        const bool need = rem > e && rr[e] < rcut2 && s < jv[e];
        ev_push<CG>(Q, need, fixed_delta(pi, pv[e], row), S, a, A.eff);
      }
      jj = jn;
    }
    __syncwarp();
    const int lane = threadIdx.x & 31;
    if (lane < Q.n) A.eff = ff_add(A.eff, pair_energy_ff<CG>(Q.q[lane], S, a));
    if (PRN && own) {
      keep_tail(kept, buf, out4, L.nslots);
      L.cnt_in[s] = kept;
      if (!CG) a.ref_p[L.perm[s]] = ref_of(pi);
    }
  } else if (s < L.nslots) {
    const auto pi = L.pos[s];
    const int row0 = ptype(pi) * a.nt;
    const int m = PRN ? L.cnt_full[s] : L.cnt[s];
    const int nch = (m + 3) >> 2;
    const int4* nb4 = reinterpret_cast<const int4*>(PRN ? L.nbr_full : L.nbr) + s;
    int4* out4 = reinterpret_cast<int4*>(L.nbr_in) + s;
    int4 buf = make_int4(s, s, s, s);
    int4 jj = make_int4(s, s, s, s);
    if (q < nch) jj = __ldcs(nb4 + size_t(q) * L.nslots);
    for (int ch = q; ch < nch; ch += TPA) {
      int4 jn = jj;
      if (ch + TPA < nch) jn = __ldcs(nb4 + size_t(ch + TPA) * L.nslots);
      const int rem = m - 4 * ch;  // >= 1
      const int j1 = rem > 1 ? jj.y : s, j2 = rem > 2 ? jj.z : s, j3 = rem > 3 ? jj.w : s;
      const auto p0 = load_pos(L.pos, jj.x);
      const auto p1 = load_pos(L.pos, j1);
      const auto p2 = load_pos(L.pos, j2);
      const auto p3 = load_pos(L.pos, j3);
      const R r0 = entry<R, CG, EV, ACC>(pi, p0, true, row0, S, a, A);
      const R r1 = entry<R, CG, EV, ACC>(pi, p1, rem > 1, row0, S, a, A);
      const R r2 = entry<R, CG, EV, ACC>(pi, p2, rem > 2, row0, S, a, A);
      const R r3 = entry<R, CG, EV, ACC>(pi, p3, rem > 3, row0, S, a, A);
      acc_chunk<ACC>(A);
      if (PRN) {
        keep_entry(r0 < L.rp2, jj.x, kept, buf, out4, L.nslots);
        keep_entry(r1 < L.rp2, j1, kept, buf, out4, L.nslots);
        keep_entry(r2 < L.rp2, j2, kept, buf, out4, L.nslots);
        keep_entry(r3 < L.rp2, j3, kept, buf, out4, L.nslots);
      }
      jj = jn;
    }
    if (PRN) {
      keep_tail(kept, buf, out4, L.nslots);
      L.cnt_in[s] = kept;
      if (!CG) a.ref_p[L.perm[s]] = ref_of(pi);
    }
  }
  if (PRN) {
    unsigned long long v[1] = {(unsigned long long)kept};
    __shared__ unsigned long long sh_k[1024 / 32];
    block_sum<unsigned long long, 1>(v, sh_k);
    if (threadIdx.x == 0) {
      atomicAdd(L.tot_in, v[0]);
      if (first_block) atomicAdd(&a.st->n_prunes, 1ull);
    }
  }
  acc_final<ACC>(A);
  if (TPA > 1) {  // every lane of the warp takes part (TPA divides 32)
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) {
      A.fx += __shfl_xor_sync(0xffffffffu, A.fx, o);
      A.fy += __shfl_xor_sync(0xffffffffu, A.fy, o);
      A.fz += __shfl_xor_sync(0xffffffffu, A.fz, o);
    }
  }
  if (s < L.nslots && q == 0) store_force(L.f_out, L.perm[s], A.fx, A.fy, A.fz);
  if (EV) {
    double accd[kNQ];
    __shared__ double sh[(1024 / 32) * kNQ];
    if constexpr (std::is_same<R, float>::value) {
      // FP32 path: warp sums in float-float (energy) and FP32 (virial: 32
      // per-thread sums of FP32 terms), FP64 across the warps only (FP64
      // arithmetic runs at a small fraction of the FP32 rate on this part).
      // Each pair's energy was counted once (queued), so it is doubled here
      // against the halving of the full-list sums below.
      ff e = A.eff;
      float w[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) w[k] = A.w[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e = ff_add(e, ff{__shfl_xor_sync(0xffffffffu, e.hi, o), __shfl_xor_sync(0xffffffffu, e.lo, o)});
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
      }
      const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      if ((threadIdx.x & 31) == 0) {
        sh[wid * kNQ] = 2.0 * (double(e.hi) + double(e.lo));
#pragma unroll
        for (int k = 0; k < 6; ++k) sh[wid * kNQ + k + 1] = double(w[k]);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kNQ; ++k) {
          double v = 0.0;
          for (int ww = 0; ww < nw; ++ww) v += sh[ww * kNQ + k];
          accd[k] = v;
        }
      }
    } else {
      // FP64 path: per-thread FP64 sums, block sum in FP64
      accd[0] = double(A.e);
#pragma unroll
      for (int k = 0; k < 6; ++k) accd[k + 1] = double(A.w[k]);
      block_sum<double, kNQ>(accd, sh);
    }
    if (threadIdx.x == 0) {
      // full lists: every pair was visited from both ends
#pragma unroll
      for (int k = 0; k < kNQ; ++k) acc_add(L.acc + k, 0.5 * accd[k]);
    }
  }
}

// Forces-only FP32 launches are held to 64 registers a thread (the occupancy
// of the walk without pruning); the pruning walk lives in the same kernel.
// FP32 energy-step launches (256-thread blocks) are held to three blocks per
// SM (80 registers; unbounded they take 95, two blocks per SM: 1.03 against
// 0.93 ms per launch at 1M atoms).
template <typename R, bool EV>
constexpr int pair_min_blocks(int bs) {
  return !std::is_same<R, float>::value ? 1 : (EV ? 3 * 256 / bs : 65536 / (64 * bs));
}

// One launch per step: with pruning on (one thread per slot) the kernel reads
// the device flags and, if a rebuild or the pruning trigger fired this step,
// walks the full lists and writes the pruned ones as it goes.
// The work of block `bid` of one system's pair launch.
template <typename R, bool EV, int TPA, int ACC>
__device__ __forceinline__ void pair_block(const PairLaunch<R>& a, int bid) {
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
      FgE* fge = reinterpret_cast<FgE*>(carve(sizeof(FgE) * nrow));
      CgE* cge = reinterpret_cast<CgE*>(carve(sizeof(CgE) * nrow));
      for (int r = threadIdx.x; r < nrow; r += blockDim.x) pack_energy_rows(a.tabd[r], fge[r], cge[r]);
      S.fge = fge;
      S.cge = cge;
      S.evq = reinterpret_cast<int4*>(carve(sizeof(int4) * kEvQueue * (blockDim.x / 32)));
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
  const bool cg = bid < a.nblk_cg;
  const int blk = cg ? bid : bid - a.nblk_cg;
  if constexpr (!std::is_same<R, float>::value && TPA > 1) {
    static_assert(!EV, "FP64 energy steps use one thread per slot");
    if (cg)
      walk_ordered<true, TPA>(a.cg, blk, S, a);
    else
      walk_ordered<false, TPA>(a.fg, blk, S, a);
  } else {
    if constexpr (TPA == 1) {
      if (a.prune_on && (*(volatile const unsigned*)a.gate & (F_REBUILD | F_PRUNE)) != 0u) {
        if (cg)
          walk<R, true, EV, 1, true, ACC>(a.cg, blk, S, a, bid == 0);
        else
          walk<R, false, EV, 1, true, ACC>(a.fg, blk, S, a, bid == 0);
        return;
      }
    }
    if (cg)
      walk<R, true, EV, TPA, false, ACC>(a.cg, blk, S, a, bid == 0);
    else
      walk<R, false, EV, TPA, false, ACC>(a.fg, blk, S, a, bid == 0);
  }
}

template <typename R, bool EV, int TPA, int BS, int ACC>
__global__ void __launch_bounds__(BS, pair_min_blocks<R, EV>(BS)) k_pair(PairLaunch<R> a) {
  // the force sum that follows may start launching once every block of this
  // grid runs (it waits for this grid to finish before reading the forces)
  grid_dependents_launch();
  pair_block<R, EV, TPA, ACC>(a, blockIdx.x);
}

// Batches (relres_batch_step): one launch over the pair work of every replica.
// Block b belongs to the replica r with off[r] <= b < off[r + 1]; its
// arguments are the replica's PairLaunch in device memory.
template <typename R, bool EV, int ACC>
__global__ void __launch_bounds__(kThreads, pair_min_blocks<R, EV>(kThreads))
    k_pair_batch(const PairLaunch<R>* __restrict__ args, const int* __restrict__ off, int nrep) {
  const int r = batch_replica(off, nrep, blockIdx.x);
  pair_block<R, EV, 1, ACC>(args[r], int(blockIdx.x) - off[r]);
}

template <typename R>
static size_t pair_smem(int nt, bool ev) {
  const size_t nrow = size_t(nt) * nt;
  auto up = [](size_t b) { return (b + 15) / 16 * 16; };
  if (std::is_same<R, float>::value)
    return up(sizeof(FgRow) * nrow) + up(sizeof(CgRow) * nrow) +
           (ev ? up(sizeof(FgE) * nrow) + up(sizeof(CgE) * nrow) + sizeof(int4) * kEvQueue * (kThreads / 32) : 0);
  return up(sizeof(PairTab<R>) * nrow);
}

// FP32 launches with the owner's force sum kept as ACC (relres_accumulation)
template <int ACC>
static cudaError_t launch_pairs_f32(relres_ctx* c, const PairLaunch<float>& a, bool ev, int grid, size_t smem) {
  if (ev) {
    k_pair<float, true, 1, kThreads, ACC><<<grid, kThreads, smem, c->stream>>>(a);
  } else {
    switch (c->pair_cfg) {
#define RELRES_PAIR_CASE(k, T, B) \
  case k:                         \
    k_pair<float, false, T, B, ACC><<<grid, B, smem, c->stream>>>(a); \
    break;
      RELRES_PAIR_CASE(0, 1, 256)
      RELRES_PAIR_CASE(1, 1, 128)
      RELRES_PAIR_CASE(2, 1, 512)
      RELRES_PAIR_CASE(3, 2, 256)
      RELRES_PAIR_CASE(4, 4, 256)
      RELRES_PAIR_CASE(5, 8, 256)
      RELRES_PAIR_CASE(6, 2, 128)
#undef RELRES_PAIR_CASE
      default:
        return cudaErrorInvalidValue;
    }
  }
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

// Arguments of one system's pair launch with `per` slots per block; returns
// the number of blocks (0: nothing to do).
// prune_in_kernel: a launch with one thread per slot prunes as it walks (else
// the lists were pruned beforehand by k_prune, or pruning is off)
template <typename R>
static int make_pair_launch(const relres_ctx* c, int which, int tpa, int per, bool prune_in_kernel,
                            PairLaunch<R>* out) {
  const double unit = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  PairLaunch<R> a{};
  a.sx = R(c->box[0] / unit);
  a.sy = R(c->box[1] / unit);
  a.sz = R(c->box[2] / unit);
  a.sxl = float(c->box[0] / unit - double(a.sx));
  a.syl = float(c->box[1] / unit - double(a.sy));
  a.szl = float(c->box[2] / unit - double(a.sz));
  a.nt = c->n_types;
  a.tab = static_cast<const PairTab<R>*>(c->d_tab);
  a.tabd = static_cast<const PairTab<double>*>(c->d_tabd);
  a.gate = &c->d_state->flags;
  a.ref_p = c->d_ref_p;
  a.st = c->d_state;
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
  const R rf = R(c->rlist_fg_cut + c->prune_delta + kPruneSlack);
  a.fg = ListWalk<R>{c->n, pfg, walk_nbr_fg(c), walk_cnt_fg(c), c->d_perm_fg,
                     static_cast<ForceOut<R>*>(c->d_f_fg), c->d_acc + kAccFg,
                     c->d_nbr_fg, c->d_cnt_fg, c->d_nbr_fg_in, c->d_cnt_fg_in, rf * rf,
                     &c->d_state->tot_in_fg};
  // without a CG list the CG walk is never entered; its pointers are stand-ins
  if (do_cg) {
    const R rc = R(c->rlist_cg_cut + c->prune_delta + kPruneSlack);
    a.cg = ListWalk<R>{c->n_h, pcg, walk_nbr_cg(c), walk_cnt_cg(c), c->d_perm_cg,
                       static_cast<ForceOut<R>*>(c->d_f_cg), c->d_acc + kAccCg,
                       c->d_nbr_cg, c->d_cnt_cg, c->d_nbr_cg_in, c->d_cnt_cg_in, rc * rc,
                       &c->d_state->tot_in_cg};
  } else {
    a.cg = a.fg;
  }
  a.prune_on = (prune_in_kernel && tpa == 1) ? 1 : 0;
  const int nb_fg = do_fg ? (c->n + per - 1) / per : 0;
  const int nb_cg = do_cg ? (c->n_h + per - 1) / per : 0;
  a.nblk_cg = nb_cg;
  *out = a;
  return nb_cg + nb_fg;
}

template <typename R>
static cudaError_t launch_pairs_t(relres_ctx* c, bool ev, int which) {
  const size_t smem = pair_smem<R>(c->n_types, ev);
  // energy steps and FP64: one thread per slot, 256 per block (32 for small
  // FP64 systems, below); forces-only FP32: the autotuned (threads per slot,
  // block size)
  int tpa = 1, bs = kThreads;
  if (std::is_same<R, float>::value && !ev) {
    tpa = kPairConfigs[c->pair_cfg].tpa;
    bs = kPairConfigs[c->pair_cfg].bs;
  }
  // FP64 runs at under 2 FMA per clock per SM on this part: a system with
  // fewer 256-slot blocks than SMs spreads its slots over more SMs in 32-thread
  // blocks, and a smaller one its forces-only walks over several threads per
  // slot (walk_ordered: the same bits as one thread)
  const bool fp64_small = !std::is_same<R, float>::value && fp64_pair_block(c) == 32;
  if (fp64_small) bs = 32;
  if (!std::is_same<R, float>::value && !ev) tpa = fp64_pair_tpa(c);
  PairLaunch<R> a;
  const int grid = make_pair_launch<R>(c, which, tpa, bs / tpa, pairs_prune(c), &a);
  if (grid == 0) return cudaSuccess;
  if constexpr (!std::is_same<R, float>::value) {
    if (fp64_small) {
      if (ev)
        k_pair<R, true, 1, 32, 0><<<grid, 32, smem, c->stream>>>(a);
      else if (tpa == kFp64SmallTpa)
        k_pair<R, false, kFp64SmallTpa, 32, 0><<<grid, 32, smem, c->stream>>>(a);
      else
        k_pair<R, false, 1, 32, 0><<<grid, 32, smem, c->stream>>>(a);
    } else if (ev) {
      k_pair<R, true, 1, kThreads, 0><<<grid, kThreads, smem, c->stream>>>(a);
    } else {
      k_pair<R, false, 1, kThreads, 0><<<grid, kThreads, smem, c->stream>>>(a);
    }
  } else {
    switch (c->force_acc) {
      case RELRES_ACC_FP32:
        return launch_pairs_f32<RELRES_ACC_FP32>(c, a, ev, grid, smem);
      case RELRES_ACC_COMPENSATED:
        return launch_pairs_f32<RELRES_ACC_COMPENSATED>(c, a, ev, grid, smem);
      case RELRES_ACC_FP64:
        return launch_pairs_f32<RELRES_ACC_FP64>(c, a, ev, grid, smem);
      default:
        return cudaErrorInvalidValue;
    }
  }
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

// ---- batches: the argument table of every replica (one thread per slot,
// 256-slot blocks, pruning in the walk) uploaded once per captured graph
template <typename R>
static cudaError_t prepare_pairs_batch_t(const std::vector<relres_ctx*>& cs, BatchLaunch* b) {
  std::vector<PairLaunch<R>> args(cs.size());
  std::vector<int> off(cs.size() + 1, 0);
  int nt_max = 1;
  for (size_t r = 0; r < cs.size(); ++r) {
    off[r + 1] = off[r] + make_pair_launch<R>(cs[r], 3, 1, kThreads, cs[r]->prune_on, &args[r]);
    nt_max = std::max(nt_max, cs[r]->n_types);
  }
  b->nblk = off.back();
  b->smem = pair_smem<R>(nt_max, false);
  b->smem_ev = pair_smem<R>(nt_max, true);
  return upload_batch(b, args.data(), sizeof(PairLaunch<R>) * args.size(), off);
}

cudaError_t prepare_pairs_batch(const std::vector<relres_ctx*>& cs, BatchLaunch* b) {
  return cs[0]->fp64 ? prepare_pairs_batch_t<double>(cs, b) : prepare_pairs_batch_t<float>(cs, b);
}

template <int ACC>
static void launch_pairs_batch_f32(cudaStream_t s, bool ev, const BatchLaunch& b, int nrep) {
  const auto* args = static_cast<const PairLaunch<float>*>(b.d_args);
  if (ev)
    k_pair_batch<float, true, ACC><<<b.nblk, kThreads, b.smem_ev, s>>>(args, b.d_off, nrep);
  else
    k_pair_batch<float, false, ACC><<<b.nblk, kThreads, b.smem, s>>>(args, b.d_off, nrep);
}

cudaError_t launch_pairs_batch(cudaStream_t s, bool fp64, int acc, bool ev, const BatchLaunch& b, int nrep) {
  if (b.nblk == 0) return cudaSuccess;
  if (fp64) {
    const auto* args = static_cast<const PairLaunch<double>*>(b.d_args);
    if (ev)
      k_pair_batch<double, true, 0><<<b.nblk, kThreads, b.smem_ev, s>>>(args, b.d_off, nrep);
    else
      k_pair_batch<double, false, 0><<<b.nblk, kThreads, b.smem, s>>>(args, b.d_off, nrep);
  } else if (acc == RELRES_ACC_FP32) {
    launch_pairs_batch_f32<RELRES_ACC_FP32>(s, ev, b, nrep);
  } else if (acc == RELRES_ACC_COMPENSATED) {
    launch_pairs_batch_f32<RELRES_ACC_COMPENSATED>(s, ev, b, nrep);
  } else {
    launch_pairs_batch_f32<RELRES_ACC_FP64>(s, ev, b, nrep);
  }
  return cudaGetLastError();
}

bool pairs_prune(const relres_ctx* c) {
  return c->prune_on && (c->fp64 ? fp64_pair_tpa(c) == 1 : kPairConfigs[c->pair_cfg].tpa == 1);
}

cudaError_t launch_pairs(relres_ctx* c, bool ev, int which) {
  return c->fp64 ? launch_pairs_t<double>(c, ev, which) : launch_pairs_t<float>(c, ev, which);
}

}  // namespace relres
