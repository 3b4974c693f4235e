// Positions, bonded terms, velocity Verlet, CSVR thermostat and reductions.
//
// State inside relres_step: positions are 64-bit periodic fixed point
// (exact, wrap-free increments; resolution L/2^64), velocities FP64.  The two
// half kicks of consecutive velocity-Verlet steps are merged: the velocity
// array holds u = v(n - 1/2) during a call, and one drift kernel per step does
//     u <- a u + b c F(n),   c = dt / (2 m),   x <- x + dt u
// with (a, b) = (1, 1) on the first step of a call (u = v(0)) and
// (alpha, alpha + 1) afterwards, alpha the CSVR factor of step n (1 for NVE):
// that is v(n) = u + c F(n), v(n) <- alpha v(n), u <- v(n) + c F(n).  The
// kinetic energy for the thermostat and the thermo output is formed from
// u + c F(n) in the finish kernel.  At the end of a call the velocities are
// returned as v(N) = a u + (b - 1) c F(N) and positions as doubles in [0, L).
//
// Bonded forces are computed per atom from the CSR list of the terms it takes
// part in (each term recomputed by each of its atoms): no atomics, and each
// term's energy is counted by its first atom.
//
// Kernel parameters are only read directly (never through a pointer or a
// reference, never indexed with a run-time index); per-type constants live in
// small device arrays.
#include "common.cuh"
#include "fbits.h"

namespace relres {

constexpr double kFtm2v = 4.184e-4;        // (kcal/mol/A)/(g/mol) -> A/fs^2
constexpr double kMvv2e = 1.0 / 4.184e-4;  // (g/mol)(A/fs)^2 -> kcal/mol

struct BoxConsts {
  double inv_l0, inv_l1, inv_l2;     // 1 / L
  double l64_0, l64_1, l64_2;        // L / 2^64
  double dts0, dts1, dts2;           // dt * 2^64 / L  (A/fs -> fixed-point units per step)
  float s32_0, s32_1, s32_2;         // L / 2^32
  double l0, l1, l2;                 // L
};

static BoxConsts box_consts(const relres_ctx* c, double dt) {
  BoxConsts b;
  b.inv_l0 = 1.0 / c->box[0];
  b.inv_l1 = 1.0 / c->box[1];
  b.inv_l2 = 1.0 / c->box[2];
  b.l64_0 = c->box[0] / 18446744073709551616.0;
  b.l64_1 = c->box[1] / 18446744073709551616.0;
  b.l64_2 = c->box[2] / 18446744073709551616.0;
  b.dts0 = dt * 18446744073709551616.0 / c->box[0];
  b.dts1 = dt * 18446744073709551616.0 / c->box[1];
  b.dts2 = dt * 18446744073709551616.0 / c->box[2];
  b.s32_0 = float(c->box[0] / 4294967296.0);
  b.s32_1 = float(c->box[1] / 4294967296.0);
  b.s32_2 = float(c->box[2] / 4294967296.0);
  b.l0 = c->box[0];
  b.l1 = c->box[1];
  b.l2 = c->box[2];
  return b;
}

static void ff_split(double v, float* hi, float* lo) {
  *hi = float(v);
  *lo = float(v - double(*hi));
}

template <typename R>
struct Sc3 {  // per-axis scale of a fixed-point difference
  R s0, s1, s2;
};

// ----------------------------------------------------------------- positions

__device__ __forceinline__ void scatter_sorted(int i, int t, unsigned long long x, unsigned long long y,
                                               unsigned long long z, const int* rank_fg,
                                               const int* rank_cg, int with_cg, int4* pos_fg,
                                               int4* pos_cg, int fp64, Pos64* pos_fg64,
                                               Pos64* pos_cg64) {
  const int4 h = make_int4(hi32(x), hi32(y), hi32(z), t);
  const int sf = rank_fg[i];
  pos_fg[sf] = h;
  if (fp64) pos_fg64[sf] = Pos64{(long long)x, (long long)y, (long long)z, t};
  if (with_cg) {
    const int sc = rank_cg[i];
    if (sc >= 0) {
      pos_cg[sc] = h;
      if (fp64) pos_cg64[sc] = Pos64{(long long)x, (long long)y, (long long)z, t};
    }
  }
}

// The same with the atom's slots given (sc < 0: no CG slot).
__device__ __forceinline__ void scatter_sorted_at(int sf, int sc, int t, unsigned long long x, unsigned long long y,
                                                  unsigned long long z, int4* pos_fg, int4* pos_cg, int fp64,
                                                  Pos64* pos_fg64, Pos64* pos_cg64) {
  const int4 h = make_int4(hi32(x), hi32(y), hi32(z), t);
  pos_fg[sf] = h;
  if (fp64) pos_fg64[sf] = Pos64{(long long)x, (long long)y, (long long)z, t};
  if (sc >= 0) {
    pos_cg[sc] = h;
    if (fp64) pos_cg64[sc] = Pos64{(long long)x, (long long)y, (long long)z, t};
  }
}

__device__ __forceinline__ bool moved_beyond(int4 ref, unsigned long long x, unsigned long long y,
                                             unsigned long long z, Sc3<float> s, float thr2) {
  const float dx = dfix32(hi32(x), ref.x, s.s0);
  const float dy = dfix32(hi32(y), ref.y, s.s1);
  const float dz = dfix32(hi32(z), ref.z, s.s2);
  return dx * dx + dy * dy + dz * dz > thr2;
}

__global__ void k_convert(int n, const double* __restrict__ pos, const int* __restrict__ type,
                          unsigned long long* __restrict__ xfx, BoxConsts b, int have_lists,
                          const int* rank_fg, const int* rank_cg, int with_cg, int4* pos_fg,
                          int4* pos_cg, int fp64, Pos64* pos_fg64, Pos64* pos_cg64, const int4* ref,
                          float thr2, const int4* ref_p, float thr2_p, int prune, DevState* st) {
  const double il0 = b.inv_l0, il1 = b.inv_l1, il2 = b.inv_l2;
  const Sc3<float> s{b.s32_0, b.s32_1, b.s32_2};
  bool rebuild = false, reprune = false, bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
    const unsigned long long ux = to_fixed(x, il0), uy = to_fixed(y, il1), uz = to_fixed(z, il2);
    xfx[3 * i] = ux;
    xfx[3 * i + 1] = uy;
    xfx[3 * i + 2] = uz;
    if (have_lists) {
      scatter_sorted(i, type[i], ux, uy, uz, rank_fg, rank_cg, with_cg, pos_fg, pos_cg, fp64, pos_fg64,
                     pos_cg64);
      rebuild |= moved_beyond(ref[i], ux, uy, uz, s, thr2);
      if (prune) reprune |= moved_beyond(ref_p[i], ux, uy, uz, s, thr2_p);
    }
  }
  if (__syncthreads_or(rebuild) && threadIdx.x == 0) atomicOr(&st->flags, F_REBUILD);
  if (__syncthreads_or(reprune) && threadIdx.x == 0) atomicOr(&st->flags, F_PRUNE);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->flags, F_NONFINITE);
}

// A 64-bit fixed-point coordinate as a double in [0, L): u L 2^-64, with u
// converted to the nearest double by integer operations (the bits of
// __ull2double_rn(u)); a product rounded up to L wraps to 0 (both positive:
// compared as bit patterns).
__device__ __forceinline__ double back_to_double(unsigned long long u, double l64, double l) {
  const double x = double_of_u64(u) * l64;
  return bits_of_double(x) >= bits_of_double(l) ? 0.0 : x;
}

// The caller's positions (and velocities, when vel is not NULL) against the
// ones the last relres_step returned, word for word: F_DIRTY / F_VDIRTY when
// any differs.
__global__ void k_check_io(int n3, const unsigned long long* __restrict__ pos,
                           const unsigned long long* __restrict__ pos_ret, const unsigned long long* __restrict__ vel,
                           const unsigned long long* __restrict__ vel_ret, DevState* st) {
  bool dp = false, dv = false;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += gridDim.x * blockDim.x) {
    dp |= pos[k] != pos_ret[k];
    if (vel != nullptr) dv |= vel[k] != vel_ret[k];
  }
  if (__syncthreads_or(dp) && threadIdx.x == 0) atomicOr(&st->flags, F_DIRTY);
  if (__syncthreads_or(dv) && threadIdx.x == 0) atomicOr(&st->flags, F_VDIRTY);
}

// ----------------------------------------------------------------- bonded

struct BondedArgs {
  const int4* bonds;
  const int4* angles;
  const int4* dihs;
  const int* dih_type;
  const double* bond_par;   // k, r0
  const double* angle_par;  // k, theta0
  const double* dih_par;    // K1..K4
  const float* bond_fpar;   // FP32 path: k, r0 (hi, lo), 0
  const float* angle_fpar;  // FP32 path: k, theta0, cos theta0 (hi, lo), sin theta0 (hi, lo), 0, 0
};

// Where the bonded terms read 64-bit fixed-point positions: the global array
// (caller order), or a segment's copy in shared memory (atoms a0, a0 + 1, ...).
struct GPos {
  const unsigned long long* x;
  __device__ __forceinline__ unsigned long long operator()(int i, int q) const { return x[3 * i + q]; }
};
struct SPos {
  const unsigned long long* s;
  int a0;
  __device__ __forceinline__ unsigned long long operator()(int i, int q) const { return s[3 * (i - a0) + q]; }
};
// global positions of atoms named by a prototype's records: atom i + off
struct GPosOff {
  const unsigned long long* x;
  int off;
  __device__ __forceinline__ unsigned long long operator()(int i, int q) const { return x[3 * (i + off) + q]; }
};

// exact 64-bit fixed-point difference a - b, scaled to Angstrom (float-float)
__device__ __forceinline__ ff ff_fixed_diff(unsigned long long a, unsigned long long b, ff scale) {
  return ff_mul(ff_from_ll((long long)(a - b)), scale);
}
template <class X>
__device__ __forceinline__ void ff_vec(const X& x, int a, int b, ff s0, ff s1, ff s2, ff v[3]) {
  v[0] = ff_fixed_diff(x(a, 0), x(b, 0), s0);
  v[1] = ff_fixed_diff(x(a, 1), x(b, 1), s1);
  v[2] = ff_fixed_diff(x(a, 2), x(b, 2), s2);
}
__device__ __forceinline__ ff ff_dot(const ff a[3], const ff b[3]) {
  return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

template <class X>
__device__ __forceinline__ void dvec(const X& x, int a, int b, Sc3<float> s, float d[3]) {
  d[0] = dfix32(hi32(x(a, 0)), hi32(x(b, 0)), s.s0);
  d[1] = dfix32(hi32(x(a, 1)), hi32(x(b, 1)), s.s1);
  d[2] = dfix32(hi32(x(a, 2)), hi32(x(b, 2)), s.s2);
}
template <class X>
__device__ __forceinline__ void dvec(const X& x, int a, int b, Sc3<double> s, double d[3]) {
  d[0] = dfix64((long long)x(a, 0), (long long)x(b, 0), s.s0);
  d[1] = dfix64((long long)x(a, 1), (long long)x(b, 1), s.s1);
  d[2] = dfix64((long long)x(a, 2), (long long)x(b, 2), s.s2);
}

template <typename R>
__device__ __forceinline__ R dot3(const R a[3], const R b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
template <typename R>
__device__ __forceinline__ void cross3(const R a[3], const R b[3], R c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// ---- one bonded term, forces on all of its atoms.  A term is evaluated once,
// by one thread, and its force on each atom (role 0..arity-1) goes to its own
// scratch slot; the finish kernel gathers each atom's slots (no atomics).
// Return value: the term energy.

template <typename R, class X>
__device__ __forceinline__ R bond_forces(const BondedArgs& B, const X& xfx, Sc3<R> sc,
                                         int4 bd, R f[2][3]) {
  R d[3];
  dvec(xfx, bd.x, bd.y, sc, d);
  const R r = sqrt(dot3(d, d));
  const R k = R(B.bond_par[2 * bd.z]), r0 = R(B.bond_par[2 * bd.z + 1]);
  const R g = R(-2) * k * (r - r0) / r;  // force on bd.x along d
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    f[0][q] = g * d[q];
    f[1][q] = -f[0][q];
  }
  return k * (r - r0) * (r - r0);
}

template <typename R, class X>
__device__ __forceinline__ R angle_forces(const BondedArgs& B, const X& xfx, Sc3<R> sc,
                                          int4 an, R f[3][3]) {
  R r1[3], r2[3];
  dvec(xfx, an.x, an.y, sc, r1);
  dvec(xfx, an.z, an.y, sc, r2);
  const R n1 = sqrt(dot3(r1, r1)), n2 = sqrt(dot3(r2, r2));
  R c = dot3(r1, r2) / (n1 * n2);
  c = c > R(1) ? R(1) : (c < R(-1) ? R(-1) : c);
  const R th = acos(c);
  R s = sqrt(R(1) - c * c);
  if (s < R(1e-6)) s = R(1e-6);
  const R k = R(B.angle_par[2 * an.w]), t0 = R(B.angle_par[2 * an.w + 1]);
  const R pref = R(2) * k * (th - t0) / s;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    f[0][q] = pref * (r2[q] / (n1 * n2) - c * r1[q] / (n1 * n1));
    f[2][q] = pref * (r1[q] / (n1 * n2) - c * r2[q] / (n2 * n2));
    f[1][q] = -(f[0][q] + f[2][q]);
  }
  return k * (th - t0) * (th - t0);
}

template <typename R, class X>
__device__ __forceinline__ R dihedral_forces(const BondedArgs& B, const X& xfx, Sc3<R> sc,
                                             int t, R f[4][3]) {
  const int4 dh = B.dihs[t];
  const double* K = B.dih_par + 4 * B.dih_type[t];
  R b1[3], b2[3], b3[3], m1[3], m2[3];
  dvec(xfx, dh.y, dh.x, sc, b1);
  dvec(xfx, dh.z, dh.y, sc, b2);
  dvec(xfx, dh.w, dh.z, sc, b3);
  cross3(b1, b2, m1);
  cross3(b2, b3, m2);
  const R nb2 = sqrt(dot3(b2, b2));
  const R phi = atan2(nb2 * dot3(b1, m2), dot3(m1, m2));
  const R k1 = R(K[0]), k2 = R(K[1]), k3 = R(K[2]), k4 = R(K[3]);
  const R dE = R(0.5) * (-k1 * sin(phi) + R(2) * k2 * sin(R(2) * phi) - R(3) * k3 * sin(R(3) * phi) +
                         R(4) * k4 * sin(R(4) * phi));
  const R mm1 = dot3(m1, m1), mm2 = dot3(m2, m2);
  const R p12 = dot3(b1, b2), p32 = dot3(b3, b2);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    // gradient of phi with respect to each atom (Blondel & Karplus form)
    const R g0 = -nb2 / mm1 * m1[q];
    const R g3 = nb2 / mm2 * m2[q];
    const R h = p12 / (mm1 * nb2) * m1[q] + p32 / (mm2 * nb2) * m2[q];
    f[0][q] = -dE * g0;
    f[1][q] = -dE * (-g0 + h);
    f[2][q] = -dE * (-g3 - h);
    f[3][q] = -dE * g3;
  }
  return R(0.5) * (k1 * (R(1) + cos(phi)) + k2 * (R(1) - cos(R(2) * phi)) + k3 * (R(1) + cos(R(3) * phi)) +
                   k4 * (R(1) - cos(R(4) * phi)));
}

// FP32 bond.  Bonds sit near their minimum with a stiff spring, so the force
// 2k (r - r0) needs r - r0 far below FP32 resolution: r is formed in
// float-float arithmetic from the exact 64-bit fixed-point difference.
template <class X>
__device__ __forceinline__ float bond_forces_ff(const BondedArgs& B, const X& xfx, ff q0,
                                                ff q1, ff q2, int4 bd, float f[2][3]) {
  const float* P = B.bond_fpar + 4 * bd.z;
  ff d[3];
  ff_vec(xfx, bd.x, bd.y, q0, q1, q2, d);
  const ff r = ff_sqrt(ff_dot(d, d));
  const float dr = ff_val(ff_sub(r, ff{P[1], P[2]}));
  const float rf = ff_val(r);
  const float g = -2.f * P[0] * dr / rf;  // force on bd.x along d
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    f[0][q] = g * ff_val(d[q]);
    f[1][q] = -f[0][q];
  }
  return P[0] * dr * dr;
}

// FP32 angle through theta - theta0 = atan2(|a x b| cos t0 - (a.b) sin t0,
// (a.b) cos t0 + |a x b| sin t0): no acos and no loss near theta0, so the
// angle error stays near 1e-7 rad (force error ~2K 1e-7 / r).
template <class X>
__device__ __forceinline__ float angle_forces_f32(const BondedArgs& B, const X& xfx,
                                                  Sc3<float> sc, int4 an, float f[3][3]) {
  const float* P = B.angle_fpar + 8 * an.w;
  float r1[3], r2[3];
  dvec(xfx, an.x, an.y, sc, r1);
  dvec(xfx, an.z, an.y, sc, r2);
  const float dot = r1[0] * r2[0] + r1[1] * r2[1] + r1[2] * r2[2];
  const float cx = r1[1] * r2[2] - r1[2] * r2[1];
  const float cy = r1[2] * r2[0] - r1[0] * r2[2];
  const float cz = r1[0] * r2[1] - r1[1] * r2[0];
  const float cn = sqrtf(cx * cx + cy * cy + cz * cz);
  const float c0 = P[2], s0 = P[4];
  const float dth = atan2f(cn * c0 - dot * s0, dot * c0 + cn * s0);
  const float q1 = r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2];
  const float q2 = r2[0] * r2[0] + r2[1] * r2[1] + r2[2] * r2[2];
  const float inv12 = rsqrtf(q1 * q2);  // 1 / (|r1| |r2|)
  const float c = dot * inv12;
  float sn = cn * inv12;
  if (sn < 1e-6f) sn = 1e-6f;
  const float pref = 2.f * P[0] * dth / sn;
  const float i11 = 1.f / q1, i22 = 1.f / q2;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    f[0][q] = pref * (r2[q] * inv12 - c * r1[q] * i11);
    f[2][q] = pref * (r1[q] * inv12 - c * r2[q] * i22);
    f[1][q] = -(f[0][q] + f[2][q]);
  }
  return P[0] * dth * dth;
}

// ----------------------------------------------------------------- finish

template <typename R>
using ForceT = typename std::conditional<std::is_same<R, float>::value, float4, double>::type;
// velocity state u: float-float pairs (FP32 path) or doubles (FP64 path), [3n]
template <typename R>
using VelT = typename std::conditional<std::is_same<R, float>::value, float2, double>::type;

// component k of u in the precision of the force arithmetic
__device__ __forceinline__ float vel_r(const float2* v, int k) {
  const float2 p = v[k];
  return __fadd_rn(p.x, p.y);
}
__device__ __forceinline__ double vel_r(const double* v, int k) { return v[k]; }
// component k of u in FP64
__device__ __forceinline__ double vel_d(const float2* v, int k) {
  const float2 p = v[k];
  return double(p.x) + double(p.y);
}
__device__ __forceinline__ double vel_d(const double* v, int k) { return v[k]; }

__device__ __forceinline__ void load_force(const float4* f, int i, float v[3]) {
  const float4 q = f[i];
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
}
__device__ __forceinline__ void load_force(const double* f, int i, double v[3]) {
  v[0] = f[3 * i];
  v[1] = f[3 * i + 1];
  v[2] = f[3 * i + 2];
}
__device__ __forceinline__ void save_force(float4* f, int i, const float v[3]) {
  f[i] = make_float4(v[0], v[1], v[2], 0.f);
}
__device__ __forceinline__ void save_force(double* f, int i, const double v[3]) {
  f[3 * i] = v[0];
  f[3 * i + 1] = v[1];
  f[3 * i + 2] = v[2];
}

template <typename R>
struct BondedKArgs {
  int nb, na, nd;  // bonds, angles, dihedrals: threads [0, nb), [nb, nb + na), [nb + na, nb + na + nd)
  BondedArgs B;
  const unsigned long long* xfx;
  Sc3<R> sc;
  float q0h, q0l, q1h, q1l, q2h, q2l;  // L / 2^64 per axis as float-float (FP32 path)
  ForceT<R>* tf;  // slots: bonds 2 per term from 0, angles 3 per term from 2 nb, dihedrals 4 from 2 nb + 3 na
  long long* acc;
};

template <int NR, typename R>
__device__ __forceinline__ void save_slots(ForceT<R>* tf, size_t base, const R f[NR][3]) {
#pragma unroll
  for (int r = 0; r < NR; ++r) save_force(tf, int(base + r), f[r]);
}

template <typename R, bool EV>
__global__ void __launch_bounds__(kThreads) k_bonded(BondedKArgs<R> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  R e = R(0);
  const Sc3<R> sc = a.sc;
  if (t < a.nb) {
    R f[2][3];
    if constexpr (std::is_same<R, float>::value)
      e = bond_forces_ff(a.B, GPos{a.xfx}, ff{a.q0h, a.q0l}, ff{a.q1h, a.q1l}, ff{a.q2h, a.q2l}, a.B.bonds[t], f);
    else
      e = bond_forces<R>(a.B, GPos{a.xfx}, sc, a.B.bonds[t], f);
    save_slots<2, R>(a.tf, 2 * size_t(t), f);
  } else if (t < a.nb + a.na) {
    const int u = t - a.nb;
    R f[3][3];
    if constexpr (std::is_same<R, float>::value)
      e = angle_forces_f32(a.B, GPos{a.xfx}, sc, a.B.angles[u], f);
    else
      e = angle_forces<R>(a.B, GPos{a.xfx}, sc, a.B.angles[u], f);
    save_slots<3, R>(a.tf, 2 * size_t(a.nb) + 3 * size_t(u), f);
  } else if (t < a.nb + a.na + a.nd) {
    const int u = t - a.nb - a.na;
    R f[4][3];
    e = dihedral_forces<R>(a.B, GPos{a.xfx}, sc, u, f);
    save_slots<4, R>(a.tf, 2 * size_t(a.nb) + 3 * size_t(a.na) + 4 * size_t(u), f);
  }
  if (EV) {
    double v[1] = {double(e)};
    __shared__ double sh[kThreads / 32];
    block_sum<double, 1>(v, sh);
    if (threadIdx.x == 0) acc_add(a.acc + kAccEb, v[0]);
  }
}

template <typename R>
struct FinishArgs {
  int n;
  const ForceT<R>* f_fg;
  const ForceT<R>* f_cg;
  int with_cg;
  const int* type;
  int hyb_mask;
  const int* inc_off;
  const int* inc;
  const ForceT<R>* tf;
  int base1, base2;    // first slot of the angles, of the dihedrals
  const VelT<R>* vel;  // u (half-step velocities) for the kinetic energy
  int with_ke;
  const double* cdt;   // per type: dt / (2 m) * ftm2v
  const double* mass;  // per type
  ForceT<R>* f_tot;
  double* f_out;       // FP64 copy in caller order
  int with_out;
  long long* acc;
  DevState* st;
};

// Total force per atom: FG part + CG part + the slots of its bonded terms;
// kinetic energy of u + c F for the thermostat.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_finish(FinishArgs<R> a) {
  R ke = R(0);
  bool bad = false;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    const int t = a.type[i];
    R f[3];
    load_force(a.f_fg, i, f);
    if (a.with_cg && ((a.hyb_mask >> t) & 1)) {
      R g[3];
      load_force(a.f_cg, i, g);
      f[0] += g[0];
      f[1] += g[1];
      f[2] += g[2];
    }
    const int k1 = a.inc_off[i + 1];
    for (int k = a.inc_off[i]; k < k1; ++k) {
      const int item = a.inc[k];
      const int kind = (item >> 30) & 3, role = (item >> 28) & 3, term = item & 0x0fffffff;
      const int slot = kind == 0 ? 2 * term + role
                                 : (kind == 1 ? a.base1 + 3 * term + role : a.base2 + 4 * term + role);
      R g[3];
      load_force(a.tf, slot, g);
      f[0] += g[0];
      f[1] += g[1];
      f[2] += g[2];
    }
    bad = !(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]));
    save_force(a.f_tot, i, f);
    if (a.with_out) {
      a.f_out[3 * i] = double(f[0]);
      a.f_out[3 * i + 1] = double(f[1]);
      a.f_out[3 * i + 2] = double(f[2]);
    }
    if (a.with_ke) {
      const R c = R(a.cdt[t]);
      R v2 = R(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const R v = vel_r(a.vel, 3 * i + q) + c * f[q];
        v2 += v * v;
      }
      ke = R(0.5 * a.mass[t] * kMvv2e) * v2;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&a.st->flags, F_NONFINITE);
  if (a.with_ke) {
    double v[1] = {double(ke)};
    __shared__ double sh[kThreads / 32];
    block_sum<double, 1>(v, sh);
    if (threadIdx.x == 0) acc_add(a.acc + kAccKe, v[0]);
  }
}

// ---- fused bonded terms + force sum, one block per segment of whole molecules
// (at most kSegAtoms atoms that no bonded term crosses).  The block evaluates
// its segment's terms into shared-memory slots (one per atom of a term), then
// each thread sums one atom's pair forces and slots: the same arithmetic as
// k_bonded + k_finish without the global slot array.

template <typename R>
struct SegArgs {
  const int* seg;  // [n_seg][kSegRec]: atoms [a0, a1), the prototype's term ranges, its first atom
  BondedArgs B;
  const unsigned long long* xfx;
  Sc3<R> sc;
  float q0h, q0l, q1h, q1l, q2h, q2l;
  const ForceT<R>* f_fg;
  const ForceT<R>* f_cg;
  int with_cg;
  const int* type;
  int hyb_mask;
  const int* inc_off;
  const int* inc;
  const VelT<R>* vel;
  int with_ke;
  const double* cdt;
  const double* mass;
  ForceT<R>* f_tot;
  double* f_out;
  int with_out;
  long long* acc;
  DevState* st;
};

template <typename R, bool EV>
__global__ void __launch_bounds__(kThreads) k_finish_seg(SegArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ForceT<R>* slot = reinterpret_cast<ForceT<R>*>(smem_raw);
  const int* g = a.seg + kSegRec * blockIdx.x;
  const int a0 = g[0], a1 = g[1], b0 = g[2], b1 = g[3], g0 = g[4], g1 = g[5], d0 = g[6], d1 = g[7], base = g[8];
  const int nb = b1 - b0, na = g1 - g0, nd = d1 - d0;
  const int base_a = 2 * nb, base_d = base_a + 3 * na;
  const Sc3<R> sc = a.sc;
  // the terms are the prototype's (atoms from `base`): shifted onto this segment
  const GPosOff xg{a.xfx, a0 - base};
  R e = R(0);
  for (int q = threadIdx.x; q < nb + na + nd; q += blockDim.x) {
    if (q < nb) {
      R f[2][3];
      if constexpr (std::is_same<R, float>::value)
        e += bond_forces_ff(a.B, xg, ff{a.q0h, a.q0l}, ff{a.q1h, a.q1l}, ff{a.q2h, a.q2l}, a.B.bonds[b0 + q], f);
      else
        e += bond_forces<R>(a.B, xg, sc, a.B.bonds[b0 + q], f);
      save_slots<2, R>(slot, 2 * size_t(q), f);
    } else if (q < nb + na) {
      const int u = q - nb;
      R f[3][3];
      if constexpr (std::is_same<R, float>::value)
        e += angle_forces_f32(a.B, xg, sc, a.B.angles[g0 + u], f);
      else
        e += angle_forces<R>(a.B, xg, sc, a.B.angles[g0 + u], f);
      save_slots<3, R>(slot, base_a + 3 * size_t(u), f);
    } else {
      const int u = q - nb - na;
      R f[4][3];
      e += dihedral_forces<R>(a.B, xg, sc, d0 + u, f);
      save_slots<4, R>(slot, base_d + 4 * size_t(u), f);
    }
  }
  if (EV) {
    double v[1] = {double(e)};
    __shared__ double sh_e[kThreads / 32];
    block_sum<double, 1>(v, sh_e);
    if (threadIdx.x == 0) acc_add(a.acc + kAccEb, v[0]);
  }
  __syncthreads();
  R ke = R(0);
  bool bad = false;
  const int i = a0 + threadIdx.x;
  if (i < a1) {
    const int t = a.type[i];
    R f[3];
    load_force(a.f_fg, i, f);
    if (a.with_cg && ((a.hyb_mask >> t) & 1)) {
      R h[3];
      load_force(a.f_cg, i, h);
      f[0] += h[0];
      f[1] += h[1];
      f[2] += h[2];
    }
    const int ip = base + threadIdx.x;  // the prototype's atom: its incident terms
    const int k1 = a.inc_off[ip + 1];
    for (int k = a.inc_off[ip]; k < k1; ++k) {
      const int item = a.inc[k];
      const int kind = (item >> 30) & 3, role = (item >> 28) & 3, term = item & 0x0fffffff;
      const int s = kind == 0 ? 2 * (term - b0) + role
                              : (kind == 1 ? base_a + 3 * (term - g0) + role : base_d + 4 * (term - d0) + role);
      R h[3];
      load_force(slot, s, h);
      f[0] += h[0];
      f[1] += h[1];
      f[2] += h[2];
    }
    bad = !(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]));
    save_force(a.f_tot, i, f);
    if (a.with_out) {
      a.f_out[3 * i] = double(f[0]);
      a.f_out[3 * i + 1] = double(f[1]);
      a.f_out[3 * i + 2] = double(f[2]);
    }
    if (a.with_ke) {
      const R c = R(a.cdt[t]);
      R v2 = R(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const R v = vel_r(a.vel, 3 * i + q) + c * f[q];
        v2 += v * v;
      }
      ke = R(0.5 * a.mass[t] * kMvv2e) * v2;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&a.st->flags, F_NONFINITE);
  if (a.with_ke) {
    double v[1] = {double(ke)};
    __shared__ double sh_k[kThreads / 32];
    block_sum<double, 1>(v, sh_k);
    if (threadIdx.x == 0) acc_add(a.acc + kAccKe, v[0]);
  }
}

// ----------------------------------------------------------------- drift

template <typename R>
struct DriftArgs {
  int n;
  VelT<R>* vel;  // u, updated
  unsigned long long* xfx;
  const ForceT<R>* f_tot;
  const int* type;
  const double* cdt;
  const float2* cdt_ff;        // FP32 path
  double dts0, dts1, dts2;
  float dts0h, dts0l, dts1h, dts1l, dts2h, dts2l;  // FP32 path: dts as float-float
  Sc3<float> s32;
  const int* rank_fg;
  const int* rank_cg;
  int with_cg;
  int4* pos_fg;
  int4* pos_cg;
  int fp64;
  Pos64* pos_fg64;
  Pos64* pos_cg64;
  const int4* ref;
  float thr2;
  const int4* ref_p;  // positions at the last pruning pass (read if prune)
  float thr2_p;
  int prune;
  int thermo_every;
  DevState* st;
};

// The inputs of one atom's drift that the force sum of the step does not
// write (the drift kernel loads them before waiting for that kernel).
template <typename R>
struct DriftIn {
  int t, sf, sc;
  VelT<R> v[3];
  unsigned long long x0[3];
  int4 ref, ref_p;
};

template <typename R>
__device__ __forceinline__ void drift_load(const DriftArgs<R>& a, int i, DriftIn<R>& in) {
  in.t = a.type[i];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    in.v[q] = a.vel[3 * i + q];
    in.x0[q] = a.xfx[3 * i + q];
  }
  in.sf = a.rank_fg[i];
  in.sc = a.with_cg ? a.rank_cg[i] : -1;
  in.ref = a.ref[i];
  in.ref_p = a.prune ? a.ref_p[i] : make_int4(0, 0, 0, 0);
}

// One atom of the drift: u <- a u + b c F, x <- x + dt u, the sorted copies
// of x, and the two displacement triggers.  Returns the new position in x.
// Every load of the atom is issued before its first store, so that no load
// waits behind a store to memory the compiler cannot tell apart from it.
template <typename R>
__device__ __forceinline__ void drift_rest(const DriftArgs<R>& a, int i, const DriftIn<R>& in,
                                           unsigned long long x[3], bool& rebuild, bool& reprune) {
  const int t = in.t;
  R f[3];
  load_force(a.f_tot, i, f);
  const VelT<R>* v = in.v;
  const unsigned long long* x0 = in.x0;
  const int sf = in.sf, sc = in.sc;
  const int4 ref = in.ref, ref_p = in.ref_p;
  VelT<R> un[3];
  if constexpr (std::is_same<R, float>::value) {
    // float-float: u <- a u + b c F and the increment u dt 2^64 / L, with no
    // FP64 instruction (FP64 runs at a small fraction of the FP32 rate here)
    const ff ca{a.st->a_hi, a.st->a_lo}, cb{a.st->b_hi, a.st->b_lo};
    const float2 cc = a.cdt_ff[t];
    const ff bc = ff_mul(cb, ff{cc.x, cc.y});
    const ff dts[3] = {ff{a.dts0h, a.dts0l}, ff{a.dts1h, a.dts1l}, ff{a.dts2h, a.dts2l}};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const ff u = ff_add(ff_mul(ca, ff{v[q].x, v[q].y}), ff_mul_f(bc, f[q]));
      un[q] = make_float2(u.hi, u.lo);
      x[q] = x0[q] + (unsigned long long)ff2ll(ff_mul(u, dts[q]));
    }
  } else {
    const double ca = a.st->a, cb = a.st->b;
    const R bc = R(cb * a.cdt[t]);
    const double dts[3] = {a.dts0, a.dts1, a.dts2};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      // the kick increment in the force's precision, accumulated in FP64
      const double u = fma(ca, v[q], double(bc * f[q]));
      un[q] = u;
      x[q] = x0[q] + (unsigned long long)__double2ll_rn(u * dts[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    a.vel[3 * i + q] = un[q];
    a.xfx[3 * i + q] = x[q];
  }
  scatter_sorted_at(sf, sc, t, x[0], x[1], x[2], a.pos_fg, a.pos_cg, a.fp64, a.pos_fg64, a.pos_cg64);
  rebuild = moved_beyond(ref, x[0], x[1], x[2], a.s32, a.thr2);
  if (a.prune) reprune = moved_beyond(ref_p, x[0], x[1], x[2], a.s32, a.thr2_p);
}

template <typename R>
__device__ __forceinline__ void drift_atom(const DriftArgs<R>& a, int i, unsigned long long x[3], bool& rebuild,
                                           bool& reprune) {
  DriftIn<R> in;
  drift_load(a, i, in);
  drift_rest(a, i, in, x, rebuild, reprune);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_drift(DriftArgs<R> a) {
  if (blockIdx.x == 0 && threadIdx.x == 0)
    a.st->ev = a.thermo_every > 0 && ((a.st->local_step + 1) % a.thermo_every) == 0;
  bool rebuild = false, reprune = false;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    unsigned long long x[3];
    drift_atom(a, i, x, rebuild, reprune);
  }
  if (__syncthreads_or(rebuild) && threadIdx.x == 0) atomicOr(&a.st->flags, F_REBUILD);
  if (__syncthreads_or(reprune) && threadIdx.x == 0) atomicOr(&a.st->flags, F_PRUNE);
}

// ---- drift + bonded terms, one block per segment of whole molecules: the
// block drifts its atoms (same arithmetic as k_drift), keeps their new
// positions in shared memory, evaluates the segment's bonded terms from there
// into shared-memory slots (same arithmetic as k_finish_seg) and writes each
// atom's bonded force (its slots summed in incident-term order).  The bonded
// forces of the new positions are thus ready before the pair kernel runs, and
// k_sum only adds the three parts.

template <typename R>
struct DriftSegArgs {
  DriftArgs<R> d;
  const int* seg;  // [n_seg][kSegRec]: atoms [a0, a1), the prototype's term ranges, its first atom
  BondedArgs B;
  Sc3<R> sc;
  float q0h, q0l, q1h, q1l, q2h, q2l;
  const int* inc_off;
  const int* inc;
  ForceT<R>* f_bond;  // caller order
  long long* acc;
};

// The work of block `bid` (segment bid) of one system's drift launch.
template <typename R, bool EV>
__device__ __forceinline__ void drift_seg_block(const DriftSegArgs<R>& a, int bid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* sx = reinterpret_cast<unsigned long long*>(smem_raw);  // [kSegAtoms][3]
  ForceT<R>* slot = reinterpret_cast<ForceT<R>*>(smem_raw + sizeof(unsigned long long) * 3 * kSegAtoms);
  const int* g = a.seg + kSegRec * bid;
  const int a0 = g[0], a1 = g[1], b0 = g[2], b1 = g[3], g0 = g[4], g1 = g[5], d0 = g[6], d1 = g[7], base = g[8];
  const int nb = b1 - b0, na = g1 - g0, nd = d1 - d0;
  const int base_a = 2 * nb, base_d = base_a + 3 * na;
  const int i = a0 + threadIdx.x;
  const int ip = base + threadIdx.x;  // the prototype's atom (its incident terms)
  // loads that do not depend on the drift, issued before it: the records of
  // this thread's first two bond/angle terms and its atom's incident-term range
  const int q0 = threadIdx.x, q1 = threadIdx.x + kSegAtoms;
  const int4 rec0 = q0 < nb ? a.B.bonds[b0 + q0] : (q0 < nb + na ? a.B.angles[g0 + q0 - nb] : make_int4(0, 0, 0, 0));
  const int4 rec1 = q1 < nb ? a.B.bonds[b0 + q1] : (q1 < nb + na ? a.B.angles[g0 + q1 - nb] : make_int4(0, 0, 0, 0));
  const int e0 = i < a1 ? a.inc_off[ip] : 0, e1 = i < a1 ? a.inc_off[ip + 1] : 0;
  DriftIn<R> in;
  if (i < a1) drift_load(a.d, i, in);
  // launched as a programmatic dependent of the force sum: everything above
  // was written before that kernel started; the total force, the thermostat
  // factor and the step counter are read after it has finished
  grid_dependency_wait();
  if (bid == 0 && threadIdx.x == 0)
    a.d.st->ev = a.d.thermo_every > 0 && ((a.d.st->local_step + 1) % a.d.thermo_every) == 0;
  bool rebuild = false, reprune = false;
  if (i < a1) {
    unsigned long long x[3];
    drift_rest(a.d, i, in, x, rebuild, reprune);
#pragma unroll
    for (int q = 0; q < 3; ++q) sx[3 * threadIdx.x + q] = x[q];
  }
  if (__syncthreads_or(rebuild) && threadIdx.x == 0) atomicOr(&a.d.st->flags, F_REBUILD);
  if (__syncthreads_or(reprune) && threadIdx.x == 0) atomicOr(&a.d.st->flags, F_PRUNE);
  // bonded terms of the segment from the new positions (the records name the
  // prototype's atoms, base .. base + a1 - a0 - 1: the same local indices)
  const SPos xs{sx, base};
  const Sc3<R> sc = a.sc;
  R e = R(0);
  for (int q = threadIdx.x, r = 0; q < nb + na + nd; q += blockDim.x, ++r) {
    if (q < nb) {
      const int4 rc = r == 0 ? rec0 : (r == 1 ? rec1 : a.B.bonds[b0 + q]);
      R f[2][3];
      if constexpr (std::is_same<R, float>::value)
        e += bond_forces_ff(a.B, xs, ff{a.q0h, a.q0l}, ff{a.q1h, a.q1l}, ff{a.q2h, a.q2l}, rc, f);
      else
        e += bond_forces<R>(a.B, xs, sc, rc, f);
      save_slots<2, R>(slot, 2 * size_t(q), f);
    } else if (q < nb + na) {
      const int u = q - nb;
      const int4 rc = r == 0 ? rec0 : (r == 1 ? rec1 : a.B.angles[g0 + u]);
      R f[3][3];
      if constexpr (std::is_same<R, float>::value)
        e += angle_forces_f32(a.B, xs, sc, rc, f);
      else
        e += angle_forces<R>(a.B, xs, sc, rc, f);
      save_slots<3, R>(slot, base_a + 3 * size_t(u), f);
    } else {
      const int u = q - nb - na;
      R f[4][3];
      e += dihedral_forces<R>(a.B, xs, sc, d0 + u, f);
      save_slots<4, R>(slot, base_d + 4 * size_t(u), f);
    }
  }
  if (EV) {
    double v[1] = {double(e)};
    __shared__ double sh_e[kThreads / 32];
    block_sum<double, 1>(v, sh_e);
    if (threadIdx.x == 0) acc_add(a.acc + kAccEb, v[0]);
  }
  __syncthreads();
  if (i < a1) {
    R f[3] = {R(0), R(0), R(0)};
    for (int k = e0; k < e1; ++k) {
      const int item = a.inc[k];
      const int kind = (item >> 30) & 3, role = (item >> 28) & 3, term = item & 0x0fffffff;
      const int s = kind == 0 ? 2 * (term - b0) + role
                              : (kind == 1 ? base_a + 3 * (term - g0) + role : base_d + 4 * (term - d0) + role);
      R h[3];
      load_force(slot, s, h);
      f[0] += h[0];
      f[1] += h[1];
      f[2] += h[2];
    }
    save_force(a.f_bond, i, f);
  }
}

template <typename R, bool EV>
__global__ void __launch_bounds__(kSegAtoms, std::is_same<R, float>::value ? 5 * kThreads / kSegAtoms : 1)
    k_drift_seg(DriftSegArgs<R> a) {
  drift_seg_block<R, EV>(a, blockIdx.x);
}

// Batches: one launch over the segments of every replica (see k_pair_batch).
template <typename R, bool EV>
__global__ void __launch_bounds__(kSegAtoms, std::is_same<R, float>::value ? 5 * kThreads / kSegAtoms : 1)
    k_drift_seg_batch(const DriftSegArgs<R>* __restrict__ args, const int* __restrict__ off, int nrep) {
  const int r = batch_replica(off, nrep, blockIdx.x);
  drift_seg_block<R, EV>(args[r], int(blockIdx.x) - off[r]);
}

// ----------------------------------------------------------------- thermostat

// splitmix64 (Steele, Lea & Flood 2014) as a counter-based generator: the
// (c+1)-th output of the sequence started at `key`.
__device__ __forceinline__ unsigned long long mix64(unsigned long long key, unsigned long long c) {
  unsigned long long z = key + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform01(unsigned long long key, unsigned long long& c) {
  // (0, 1]: top 53 bits plus one ulp
  return (double(mix64(key, c++) >> 11) + 1.0) * 1.1102230246251565e-16;
}
__device__ double gauss(unsigned long long key, unsigned long long& c) {
  const double u1 = uniform01(key, c), u2 = uniform01(key, c);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
// Marsaglia & Tsang (2000) gamma(shape, 1) for shape >= 1
__device__ double gamma_mt(double shape, unsigned long long key, unsigned long long& c) {
  const double d = shape - 1.0 / 3.0, k = 1.0 / sqrt(9.0 * d);
  for (int it = 0; it < 1000; ++it) {
    const double x = gauss(key, c);
    double v = 1.0 + k * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    if (log(uniform01(key, c)) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
  }
  return d;
}
// Bussi-Donadio-Parrinello (2007) velocity rescaling.  The two random
// numbers of step `step` (a normal deviate r1 and a chi-square deviate s with
// n_f - 1 degrees of freedom, drawn as twice a gamma(n_f/2 - 1/2) deviate)
// depend only on the seed and the step, so a block of steps has them drawn
// in parallel ahead of time.
__device__ void csvr_draws(double n_f, unsigned long long seed, unsigned long long step, double& r1,
                           double& s) {
  unsigned long long c = step << 20;
  r1 = gauss(seed, c);
  s = 2.0 * gamma_mt(0.5 * (n_f - 1.0), seed, c);
}
// e = exp(-dt / tau), computed once per call on the host
__device__ double csvr_alpha(double ke, double e, double n_f, double kt, double r1, double s) {
  const double kn = ke + (1.0 - e) * (kt / n_f * (r1 * r1 + s) - ke) +
                    2.0 * r1 * sqrt(e * (1.0 - e) * ke * kt / n_f);
  return sqrt(kn / ke);
}

// Draws for the steps st->step + k, k < count (one thread each).
__global__ void k_csvr_draws(double n_f, unsigned long long seed, int count, const DevState* st,
                             double* draws) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  double r1, s;
  csvr_draws(n_f, seed, st->step + (unsigned long long)k, r1, s);
  draws[2 * k] = r1;
  draws[2 * k + 1] = s;
}

// End of a step (one thread): thermostat factor from the kinetic energy,
// thermo row on energy steps, counters, and the accumulators cleared for the
// next step.  `draw` points at this step's (r1, s).  The accumulators are read
// through volatile loads (other blocks of the calling kernel added to them).
__device__ void end_of_step(volatile long long* acc, const StepParams& sp, DevState* st, double r1, double s) {
  const bool ev = st->ev != 0;
  const double ke = double(acc[kAccKe]) / kFix;
  double alpha = 1.0;
  if (sp.t_target > 0.0 && ke > 0.0) alpha = csvr_alpha(ke, sp.csvr_e, sp.n_f, sp.kt, r1, s);
  st->alpha = alpha;
  st->a = alpha;
  st->b = alpha + 1.0;
  st->a_hi = float(alpha);
  st->a_lo = float(alpha - double(st->a_hi));
  st->b_hi = float(alpha + 1.0);
  st->b_lo = float((alpha + 1.0) - double(st->b_hi));
  double* thermo = sp.thermo;
  if (ev && sp.thermo_every > 0) {
    double* row = thermo + (size_t)st->thermo_row * RELRES_THERMO_COLS;
    row[0] = double(acc[kAccFg]) / kFix;
    row[1] = double(acc[kAccCg]) / kFix;
    row[2] = double(acc[kAccEb]) / kFix;
    row[3] = ke * alpha * alpha;
#pragma unroll
    for (int q = 1; q < kNQ; ++q) row[3 + q] = double(acc[kAccFg + q] + acc[kAccCg + q]) / kFix;
    st->thermo_row += 1;
  }
#pragma unroll
  for (int q = 0; q < kNAcc; ++q) acc[q] = 0;
  st->local_step += 1;
  st->step += 1;
  if (st->flags & F_REBUILD) {
    st->n_builds += 1;
    st->flags &= ~F_REBUILD;
  }
  st->flags &= ~F_PRUNE;  // a pruning pass ran this step if it was set
}

__global__ void k_thermo(long long* acc, StepParams sp, DevState* st, const double* draw) {
  end_of_step(acc, sp, st, sp.t_target > 0.0 ? draw[0] : 0.0, sp.t_target > 0.0 ? draw[1] : 0.0);
}

// ---- end of a step with bonded forces from k_drift_seg: per atom the total
// force F = F_FG + F_CG + F_bonded and the kinetic energy of u + c F; the last
// block to finish (a ticket counter after a memory fence) runs the thermostat
// and the step bookkeeping of k_thermo, so the step needs no separate launch.

template <typename R>
struct SumArgs {
  int n;
  const ForceT<R>* f_fg;
  const ForceT<R>* f_cg;
  int with_cg;
  const ForceT<R>* f_bond;
  const int* type;
  int hyb_mask;
  const VelT<R>* vel;
  const double* cdt;
  const float2* cdt_ff;
  const double* mass;
  const float* kec;
  ForceT<R>* f_tot;
  long long* acc;
  DevState* st;
  StepParams sp;
  const double* draw;
};

// The inputs of one atom of the force sum.
template <typename R>
struct SumIn {
  int t;
  R f[3], h[3], b[3];
  VelT<R> v[3];
};

template <typename R>
__device__ __forceinline__ void sum_load(const SumArgs<R>& a, int i, SumIn<R>& in) {
  in.t = a.type[i];
  load_force(a.f_fg, i, in.f);
  // the CG part is zero for ordinary atoms (never written): loaded without
  // waiting for the type, added only for hybrids
  if (a.with_cg) load_force(a.f_cg, i, in.h);
  load_force(a.f_bond, i, in.b);
#pragma unroll
  for (int q = 0; q < 3; ++q) in.v[q] = a.vel[3 * i + q];
}

// F = F_FG + F_CG + F_bonded of one atom, stored; returns the kinetic energy
// of u + c F.
template <typename R>
__device__ __forceinline__ R sum_atom(const SumArgs<R>& a, int i, SumIn<R>& in, bool& bad) {
  const int t = in.t;
  R* f = in.f;
  if (a.with_cg && ((a.hyb_mask >> t) & 1)) {
    f[0] += in.h[0];
    f[1] += in.h[1];
    f[2] += in.h[2];
  }
  f[0] += in.b[0];
  f[1] += in.b[1];
  f[2] += in.b[2];
  bad |= !(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]));
  save_force(a.f_tot, i, f);
  R c, kc;
  if constexpr (std::is_same<R, float>::value) {
    c = a.cdt_ff[t].x;
    kc = a.kec[t];
  } else {
    c = a.cdt[t];
    kc = 0.5 * a.mass[t] * kMvv2e;
  }
  R v2 = R(0);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const R v = vel_r(&in.v[q], 0) + c * f[q];
    v2 += v * v;
  }
  return kc * v2;
}

// grid-stride over the nblk blocks of one system (a few blocks per SM), one
// kinetic-energy atomic and one ticket per block; step k of the block of
// steps (its thermostat draws)
template <typename R>
__device__ __forceinline__ void sum_block(const SumArgs<R>& a, int bid, int nblk, int k) {
  // this step's thermostat draws, read early (the last block uses them)
  double r1 = 0.0, rs = 0.0;
  if (threadIdx.x == 0 && a.sp.t_target > 0.0) {
    r1 = a.draw[2 * k];
    rs = a.draw[2 * k + 1];
  }
  // launched as a programmatic dependent of the pair kernel: wait for its
  // forces, then let the next drift launch (its early loads read nothing that
  // this kernel or the pair kernel writes after this point)
  grid_dependency_wait();
  grid_dependents_launch();
  R ke = R(0);  // a few atoms per thread
  bool bad = false;
  const int stride = nblk * blockDim.x;
  int i = bid * blockDim.x + threadIdx.x;
  for (; i + stride < a.n; i += 2 * stride) {  // two atoms in flight: both loaded before either store
    SumIn<R> in0, in1;
    sum_load(a, i, in0);
    sum_load(a, i + stride, in1);
    const R k0 = sum_atom(a, i, in0, bad);
    const R k1 = sum_atom(a, i + stride, in1, bad);
    ke += k0 + k1;
  }
  if (i < a.n) {
    SumIn<R> in;
    sum_load(a, i, in);
    ke += sum_atom(a, i, in, bad);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&a.st->flags, F_NONFINITE);
  double v[1] = {double(ke)};
  __shared__ double sh_k[kThreads / 32];
  block_sum<double, 1>(v, sh_k);
  if (threadIdx.x == 0) {
    acc_add(a.acc + kAccKe, v[0]);
    __threadfence();
    const unsigned ticket = atomicAdd(&a.st->done_blocks, 1u);
    if (ticket == unsigned(nblk - 1)) {
      __threadfence();
      a.st->done_blocks = 0u;
      end_of_step(a.acc, a.sp, a.st, r1, rs);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_sum(SumArgs<R> a, int k) {
  sum_block<R>(a, blockIdx.x, gridDim.x, k);
}

// Batches: one launch over every replica (see k_pair_batch); replica r's
// blocks count their own tickets, so its last block runs its thermostat.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_sum_batch(const SumArgs<R>* __restrict__ args,
                                                        const int* __restrict__ off, int nrep, int k) {
  const int r = batch_replica(off, nrep, blockIdx.x);
  sum_block<R>(args[r], int(blockIdx.x) - off[r], off[r + 1] - off[r], k);
}

// Energies and virial of relres_compute (one thread); clears the accumulators.
__global__ void k_reduce_out(long long* acc, double* energy, int with_e, double* virial, int with_w) {
  const double efg = double(acc[kAccFg]) / kFix, ecg = double(acc[kAccCg]) / kFix;
  const double eb = double(acc[kAccEb]) / kFix;
  if (with_e) {
    energy[0] = efg;
    energy[1] = ecg;
    energy[2] = eb;
    energy[3] = efg + ecg + eb;
  }
  if (with_w)
#pragma unroll
    for (int q = 1; q < kNQ; ++q) virial[q - 1] = double(acc[kAccFg + q] + acc[kAccCg + q]) / kFix;
#pragma unroll
  for (int q = 0; q < kNAcc; ++q) acc[q] = 0;
}

// Start of a relres_step call: its step and thermo-row counters, and (unless
// the call continues the velocity state of the last one) the factors of the
// first drift for velocities read from the caller, u = v: a = b = 1.
__global__ void k_call_start(DevState* st, int reset_ab) {
  if (reset_ab) {
    st->a = 1.0;
    st->b = 1.0;
    st->a_hi = 1.f;
    st->a_lo = 0.f;
    st->b_hi = 1.f;
    st->b_lo = 0.f;
  }
  st->local_step = 0;
  st->thermo_row = 0;
  st->ev = 0;
}

__global__ void k_flags_and(DevState* st, unsigned keep) { st->flags &= keep; }

// FP32 path: caller's FP64 velocities -> float-float state
__global__ void k_vel_in(int n3, const double* __restrict__ vel, float2* __restrict__ uff) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += gridDim.x * blockDim.x) {
    const double v = vel[k];
    const float hi = float(v);
    uff[k] = make_float2(hi, float(v - double(hi)));
  }
}

template <typename R>
__global__ void k_finish_md(int n, const DevState* st, const VelT<R>* vel_u,
                            const ForceT<R>* __restrict__ f_tot, const int* __restrict__ type,
                            const double* __restrict__ cdt, const float2* __restrict__ cdt_ff,
                            const unsigned long long* __restrict__ xfx, BoxConsts b, double* vel_out,
                            double* __restrict__ pos_out, double* __restrict__ pos_ret, double* __restrict__ vel_ret) {
  const double a0 = b.l64_0, a1 = b.l64_1, a2 = b.l64_2, l0 = b.l0, l1 = b.l1, l2 = b.l2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int t = type[i];
    R f[3];
    load_force(f_tot, i, f);
    double v[3];
    if constexpr (std::is_same<R, float>::value) {
      // v = a u + (b - 1) c F in float-float, returned as the double nearest
      // to hi + lo: the parts converted exactly with integer operations, one
      // FP64 addition
      const ff ca{st->a_hi, st->a_lo};
      const ff cb1 = ff_add(ff{st->b_hi, st->b_lo}, ff{-1.f, 0.f});
      const float2 cc = cdt_ff[t];
      const ff cbc = ff_mul(cb1, ff{cc.x, cc.y});
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float2 u = vel_u[3 * i + q];
        const ff w = ff_add(ff_mul(ca, ff{u.x, u.y}), ff_mul_f(cbc, f[q]));
        v[q] = double_of_float(w.hi) + double_of_float(w.lo);
      }
    } else {
      const double ca = st->a, cb1 = st->b - 1.0;
      const R c = R(cb1 * cdt[t]);
#pragma unroll
      for (int q = 0; q < 3; ++q) v[q] = fma(ca, vel_d(vel_u, 3 * i + q), double(c * f[q]));
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      vel_out[3 * i + q] = v[q];
      if (vel_ret) vel_ret[3 * i + q] = v[q];
    }
    const double x[3] = {back_to_double(xfx[3 * i], a0, l0), back_to_double(xfx[3 * i + 1], a1, l1),
                         back_to_double(xfx[3 * i + 2], a2, l2)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      pos_out[3 * i + q] = x[q];
      if (pos_ret) pos_ret[3 * i + q] = x[q];
    }
  }
}

// ----------------------------------------------------------------- launchers

static int grid_for(int n) {
  const int b = (n + kThreads - 1) / kThreads;
  return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

static float trigger_thr2(const relres_ctx* c) {
  double skin = c->prm.skin;
  if (c->has_cg && c->n_h > 0 && c->skin_cg < skin) skin = c->skin_cg;
  const double h = 0.5 * skin;
  return float(h * h);
}

// pruning trigger: half the pruning margin
static float prune_thr2(const relres_ctx* c) {
  const double h = 0.5 * c->prune_delta;
  return float(h * h);
}

static Sc3<float> s32_of(const relres_ctx* c) {
  return Sc3<float>{float(c->box[0] / 4294967296.0), float(c->box[1] / 4294967296.0),
                    float(c->box[2] / 4294967296.0)};
}

cudaError_t upload_type_consts(relres_ctx* c, double dt) {
  if (c->consts_dt == dt) return cudaSuccess;  // already there (reset by relres_set_topology)
  std::vector<float2> cff(size_t(c->n_types));
  std::vector<float> kec(size_t(c->n_types));
  for (int k = 0; k < c->n_types; ++k) {
    c->h_cdt[k] = 0.5 * dt / c->mass_by_type[k] * kFtm2v;
    float hi, lo;
    ff_split(c->h_cdt[k], &hi, &lo);
    cff[size_t(k)] = make_float2(hi, lo);
    kec[size_t(k)] = float(0.5 * c->mass_by_type[k] * kMvv2e);
  }
  cudaError_t e = cudaMemcpyAsync(c->d_cdt, c->h_cdt.data(), sizeof(double) * c->n_types, cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_cdt_ff, cff.data(), sizeof(float2) * c->n_types, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_kec, kec.data(), sizeof(float) * c->n_types, cudaMemcpyHostToDevice, c->stream);
  // the host vectors must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) c->consts_dt = dt;
  return e;
}

cudaError_t launch_vel_in(relres_ctx* c, const double* d_vel) {
  if (c->fp64) return cudaSuccess;
  const int n3 = 3 * c->n;
  k_vel_in<<<std::max(1, std::min((n3 + kThreads - 1) / kThreads, 152 * 8)), kThreads, 0, c->stream>>>(
      n3, d_vel, c->d_uff);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

static Pos64* p64(relres_ctx* c, Pos64* p) { return c->fp64 ? p : static_cast<Pos64*>(c->d_dummy); }

cudaError_t launch_convert(relres_ctx* c, const double* d_pos) {
  const BoxConsts b = box_consts(c, 0.0);
  k_convert<<<grid_for(c->n), kThreads, 0, c->stream>>>(
      c->n, d_pos, c->d_type, c->d_xfx, b, c->have_lists ? 1 : 0, c->d_rank_fg, c->d_rank_cg,
      (c->has_cg && c->n_h > 0) ? 1 : 0, c->d_pos_fg, c->d_pos_cg, c->fp64 ? 1 : 0, p64(c, c->d_pos_fg64),
      p64(c, c->d_pos_cg64), c->d_ref, trigger_thr2(c), c->prune_on ? c->d_ref_p : c->d_ref, prune_thr2(c),
      c->prune_on ? 1 : 0, c->d_state);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_check_io(relres_ctx* c, const double* d_pos, const double* d_vel) {
  const int n3 = 3 * c->n;
  k_check_io<<<std::max(1, std::min((n3 + kThreads - 1) / kThreads, 152 * 8)), kThreads, 0, c->stream>>>(
      n3, reinterpret_cast<const unsigned long long*>(d_pos), reinterpret_cast<const unsigned long long*>(c->d_pos_ret),
      reinterpret_cast<const unsigned long long*>(d_vel), reinterpret_cast<const unsigned long long*>(c->d_vel_ret),
      c->d_state);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

static BondedArgs bonded_args(const relres_ctx* c) {
  return BondedArgs{c->d_bonds,     c->d_angles,    c->d_dihs,     c->d_dih_type, c->d_bond_par,
                    c->d_angle_par, c->d_dih_par,   c->d_bond_fpar, c->d_angle_fpar};
}


template <typename R>
static cudaError_t launch_bonded_t(relres_ctx* c, bool ev) {
  const int nt = c->n_bonds + c->n_angles + c->n_dih;
  if (nt == 0) return cudaSuccess;
  const double k = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  BondedKArgs<R> a{};
  a.nb = c->n_bonds;
  a.na = c->n_angles;
  a.nd = c->n_dih;
  a.B = bonded_args(c);
  a.xfx = c->d_xfx;
  a.sc = Sc3<R>{R(c->box[0] / k), R(c->box[1] / k), R(c->box[2] / k)};
  ff_split(c->box[0] / 18446744073709551616.0, &a.q0h, &a.q0l);
  ff_split(c->box[1] / 18446744073709551616.0, &a.q1h, &a.q1l);
  ff_split(c->box[2] / 18446744073709551616.0, &a.q2h, &a.q2l);
  a.tf = static_cast<ForceT<R>*>(c->d_tf);
  a.acc = c->d_acc;
  const int nblk = (nt + kThreads - 1) / kThreads;
  if (ev)
    k_bonded<R, true><<<nblk, kThreads, 0, c->stream>>>(a);
  else
    k_bonded<R, false><<<nblk, kThreads, 0, c->stream>>>(a);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_finish_t(relres_ctx* c, double* d_forces_out, const double* vel) {
  const int with_cg = (c->has_cg && c->n_h > 0) ? 1 : 0;
  FinishArgs<R> a{c->n,
                  static_cast<const ForceT<R>*>(c->d_f_fg),
                  static_cast<const ForceT<R>*>(c->d_f_cg),
                  with_cg,
                  c->d_type,
                  c->hyb_mask,
                  c->d_inc_off,
                  c->d_inc,
                  static_cast<const ForceT<R>*>(c->d_tf),
                  2 * c->n_bonds,
                  2 * c->n_bonds + 3 * c->n_angles,
                  vel ? static_cast<const VelT<R>*>(vel_state(c, const_cast<double*>(vel)))
                      : static_cast<const VelT<R>*>(c->d_dummy),
                  vel ? 1 : 0,
                  c->d_cdt,
                  c->d_mass,
                  static_cast<ForceT<R>*>(c->d_f_tot),
                  d_forces_out ? d_forces_out : static_cast<double*>(c->d_dummy),
                  d_forces_out ? 1 : 0,
                  c->d_acc,
                  c->d_state};
  k_finish<R><<<(c->n + kThreads - 1) / kThreads, kThreads, 0, c->stream>>>(a);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_finish_seg_t(relres_ctx* c, bool ev, double* d_forces_out, const double* vel) {
  const double k = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  SegArgs<R> a{};
  a.seg = c->d_seg;
  a.B = bonded_args(c);
  a.xfx = c->d_xfx;
  a.sc = Sc3<R>{R(c->box[0] / k), R(c->box[1] / k), R(c->box[2] / k)};
  ff_split(c->box[0] / 18446744073709551616.0, &a.q0h, &a.q0l);
  ff_split(c->box[1] / 18446744073709551616.0, &a.q1h, &a.q1l);
  ff_split(c->box[2] / 18446744073709551616.0, &a.q2h, &a.q2l);
  a.f_fg = static_cast<const ForceT<R>*>(c->d_f_fg);
  a.f_cg = static_cast<const ForceT<R>*>(c->d_f_cg);
  a.with_cg = (c->has_cg && c->n_h > 0) ? 1 : 0;
  a.type = c->d_type;
  a.hyb_mask = c->hyb_mask;
  a.inc_off = c->d_inc_off;
  a.inc = c->d_inc;
  a.vel = vel ? static_cast<const VelT<R>*>(vel_state(c, const_cast<double*>(vel)))
              : static_cast<const VelT<R>*>(c->d_dummy);
  a.with_ke = vel ? 1 : 0;
  a.cdt = c->d_cdt;
  a.mass = c->d_mass;
  a.f_tot = static_cast<ForceT<R>*>(c->d_f_tot);
  a.f_out = d_forces_out ? d_forces_out : static_cast<double*>(c->d_dummy);
  a.with_out = d_forces_out ? 1 : 0;
  a.acc = c->d_acc;
  a.st = c->d_state;
  const size_t smem = size_t(c->seg_slots) * (std::is_same<R, float>::value ? 16 : 24);
  if (ev)
    k_finish_seg<R, true><<<c->n_seg, kThreads, smem, c->stream>>>(a);
  else
    k_finish_seg<R, false><<<c->n_seg, kThreads, smem, c->stream>>>(a);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_finish(relres_ctx* c, bool ev, double* d_forces_out, const double* d_vel) {
  if (c->seg_ok && c->use_seg)
    return c->fp64 ? launch_finish_seg_t<double>(c, ev, d_forces_out, d_vel)
                   : launch_finish_seg_t<float>(c, ev, d_forces_out, d_vel);
  if (c->fp64) {
    const cudaError_t e = launch_bonded_t<double>(c, ev);
    return e != cudaSuccess ? e : launch_finish_t<double>(c, d_forces_out, d_vel);
  }
  const cudaError_t e = launch_bonded_t<float>(c, ev);
  return e != cudaSuccess ? e : launch_finish_t<float>(c, d_forces_out, d_vel);
}

cudaError_t launch_reduce_out(relres_ctx* c, double* d_energy, double* d_virial) {
  double* dd = static_cast<double*>(c->d_dummy);
  k_reduce_out<<<1, 1, 0, c->stream>>>(c->d_acc, d_energy ? d_energy : dd, d_energy ? 1 : 0,
                                       d_virial ? d_virial : dd, d_virial ? 1 : 0);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_csvr_draws(relres_ctx* c, const StepParams& sp, int count) {
  if (!(sp.t_target > 0.0) || count <= 0) return cudaSuccess;
  k_csvr_draws<<<(count + 127) / 128, 128, 0, c->stream>>>(sp.n_f, sp.seed, count, c->d_state, c->d_draws);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

template <typename R>
static DriftArgs<R> drift_args(relres_ctx* c, const StepParams& sp, double* d_vel) {
  const bool cg = c->has_cg && c->n_h > 0;
  const BoxConsts b = box_consts(c, sp.dt);
  float h[6];
  ff_split(b.dts0, &h[0], &h[1]);
  ff_split(b.dts1, &h[2], &h[3]);
  ff_split(b.dts2, &h[4], &h[5]);
  return DriftArgs<R>{c->n,
                      static_cast<VelT<R>*>(vel_state(c, d_vel)),
                      c->d_xfx,
                      static_cast<const ForceT<R>*>(c->d_f_tot),
                      c->d_type,
                      c->d_cdt,
                      c->d_cdt_ff,
                      b.dts0,
                      b.dts1,
                      b.dts2,
                      h[0],
                      h[1],
                      h[2],
                      h[3],
                      h[4],
                      h[5],
                      s32_of(c),
                      c->d_rank_fg,
                      c->d_rank_cg,
                      cg ? 1 : 0,
                      c->d_pos_fg,
                      c->d_pos_cg,
                      c->fp64 ? 1 : 0,
                      p64(c, c->d_pos_fg64),
                      p64(c, c->d_pos_cg64),
                      c->d_ref,
                      trigger_thr2(c),
                      c->prune_on ? c->d_ref_p : c->d_ref,
                      prune_thr2(c),
                      c->prune_on ? 1 : 0,
                      sp.thermo_every,
                      c->d_state};
}

template <typename R>
static DriftSegArgs<R> drift_seg_args(relres_ctx* c, const StepParams& sp, double* d_vel) {
  const double k = std::is_same<R, float>::value ? 4294967296.0 : 18446744073709551616.0;
  DriftSegArgs<R> a{};
  a.d = drift_args<R>(c, sp, d_vel);
  a.seg = c->d_seg;
  a.B = bonded_args(c);
  a.sc = Sc3<R>{R(c->box[0] / k), R(c->box[1] / k), R(c->box[2] / k)};
  ff_split(c->box[0] / 18446744073709551616.0, &a.q0h, &a.q0l);
  ff_split(c->box[1] / 18446744073709551616.0, &a.q1h, &a.q1l);
  ff_split(c->box[2] / 18446744073709551616.0, &a.q2h, &a.q2l);
  a.inc_off = c->d_inc_off;
  a.inc = c->d_inc;
  a.f_bond = static_cast<ForceT<R>*>(c->d_f_bond);
  a.acc = c->d_acc;
  return a;
}

template <typename R>
static size_t drift_seg_smem(const relres_ctx* c) {
  return sizeof(unsigned long long) * 3 * kSegAtoms + size_t(c->seg_slots) * (std::is_same<R, float>::value ? 16 : 24);
}

// A launch that may overlap the tail of the previous kernel of the stream
// (programmatic dependent launch) when pdl is set: the kernel waits for that
// kernel (grid_dependency_wait) before reading what it writes.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Programmatic dependent launches only without timing events between the
// kernels (an event between them would stand in the way).
static bool pdl_ok(const relres_ctx* c) { return c->use_pdl && !c->timing; }

template <typename R>
static cudaError_t launch_drift_t(relres_ctx* c, const StepParams& sp, double* d_vel, bool ev, bool after_sum) {
  if (step_segments(c)) {
    const DriftSegArgs<R> a = drift_seg_args<R>(c, sp, d_vel);
    const size_t smem = drift_seg_smem<R>(c);
    // after the force sum of the previous step: overlap its tail
    const bool pdl = after_sum && pdl_ok(c);
    const cudaError_t e = ev ? launch_pdl(pdl, k_drift_seg<R, true>, c->n_seg, kSegAtoms, smem, c->stream, a)
                             : launch_pdl(pdl, k_drift_seg<R, false>, c->n_seg, kSegAtoms, smem, c->stream, a);
    if (e != cudaSuccess) return e;
  } else {
    k_drift<R><<<(c->n + kThreads - 1) / kThreads, kThreads, 0, c->stream>>>(drift_args<R>(c, sp, d_vel));
  }
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_drift(relres_ctx* c, const StepParams& sp, double* d_vel, bool ev, bool after_sum) {
  return c->fp64 ? launch_drift_t<double>(c, sp, d_vel, ev, after_sum)
                 : launch_drift_t<float>(c, sp, d_vel, ev, after_sum);
}

// blocks of the force sum: one wave of resident blocks (56 registers a
// thread: four blocks per SM); batches give each replica the same blocks, so
// its kinetic-energy partial sums, and with them its trajectory, are the same
// bits as stepping it alone
static int sum_blocks(const relres_ctx* c) { return std::max(1, std::min((c->n + kThreads - 1) / kThreads, 152 * 4)); }

template <typename R>
static SumArgs<R> sum_args(relres_ctx* c, const StepParams& sp, const double* d_vel) {
  SumArgs<R> a{};
  a.n = c->n;
  a.f_fg = static_cast<const ForceT<R>*>(c->d_f_fg);
  a.f_cg = static_cast<const ForceT<R>*>(c->d_f_cg);
  a.with_cg = (c->has_cg && c->n_h > 0) ? 1 : 0;
  a.f_bond = static_cast<const ForceT<R>*>(c->d_f_bond);
  a.type = c->d_type;
  a.hyb_mask = c->hyb_mask;
  a.vel = static_cast<const VelT<R>*>(vel_state(c, const_cast<double*>(d_vel)));
  a.cdt = c->d_cdt;
  a.cdt_ff = c->d_cdt_ff;
  a.mass = c->d_mass;
  a.kec = c->d_kec;
  a.f_tot = static_cast<ForceT<R>*>(c->d_f_tot);
  a.acc = c->d_acc;
  a.st = c->d_state;
  a.sp = sp;
  if (a.sp.thermo == nullptr) {
    a.sp.thermo = static_cast<double*>(c->d_dummy);
    a.sp.thermo_every = 0;
  }
  a.draw = c->d_draws;
  return a;
}

template <typename R>
static cudaError_t launch_sum_t(relres_ctx* c, const StepParams& sp, int k, const double* d_vel) {
  const SumArgs<R> a = sum_args<R>(c, sp, d_vel);
  // after the pair kernel: overlap its tail
  const cudaError_t e = launch_pdl(pdl_ok(c), k_sum<R>, sum_blocks(c), kThreads, 0, c->stream, a, k);
  if (e != cudaSuccess) return e;
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_end_of_step(relres_ctx* c, const StepParams& sp, int k, bool ev, double* d_vel) {
  if (step_segments(c))
    return c->fp64 ? launch_sum_t<double>(c, sp, k, d_vel) : launch_sum_t<float>(c, sp, k, d_vel);
  cudaError_t e = launch_finish(c, ev, nullptr, d_vel);
  return e != cudaSuccess ? e : launch_thermo(c, sp, k);
}

cudaError_t launch_thermo(relres_ctx* c, const StepParams& sp, int k) {
  StepParams q = sp;
  if (q.thermo == nullptr) {
    q.thermo = static_cast<double*>(c->d_dummy);
    q.thermo_every = 0;
  }
  k_thermo<<<1, 1, 0, c->stream>>>(c->d_acc, q, c->d_state, c->d_draws + 2 * k);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_call_start(relres_ctx* c, bool reset_ab) {
  k_call_start<<<1, 1, 0, c->stream>>>(c->d_state, reset_ab ? 1 : 0);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_flags_and(relres_ctx* c, unsigned keep) {
  k_flags_and<<<1, 1, 0, c->stream>>>(c->d_state, keep);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

// ---- batches (relres_batch_step): argument tables of every replica
template <typename R>
static cudaError_t prepare_drift_batch_t(const std::vector<relres_ctx*>& cs, const std::vector<StepParams>& sp,
                                         double* const* d_vel, BatchLaunch* b) {
  std::vector<DriftSegArgs<R>> args(cs.size());
  std::vector<int> off(cs.size() + 1, 0);
  size_t smem = 0;
  for (size_t r = 0; r < cs.size(); ++r) {
    args[r] = drift_seg_args<R>(cs[r], sp[r], d_vel[r]);
    off[r + 1] = off[r] + cs[r]->n_seg;
    smem = std::max(smem, drift_seg_smem<R>(cs[r]));
  }
  b->nblk = off.back();
  b->smem = b->smem_ev = smem;
  return upload_batch(b, args.data(), sizeof(DriftSegArgs<R>) * args.size(), off);
}

cudaError_t prepare_drift_batch(const std::vector<relres_ctx*>& cs, const std::vector<StepParams>& sp,
                                double* const* d_vel, BatchLaunch* b) {
  return cs[0]->fp64 ? prepare_drift_batch_t<double>(cs, sp, d_vel, b) : prepare_drift_batch_t<float>(cs, sp, d_vel, b);
}

template <typename R>
static void launch_drift_batch_t(cudaStream_t s, bool ev, const BatchLaunch& b, int nrep) {
  const auto* args = static_cast<const DriftSegArgs<R>*>(b.d_args);
  if (ev)
    k_drift_seg_batch<R, true><<<b.nblk, kSegAtoms, b.smem, s>>>(args, b.d_off, nrep);
  else
    k_drift_seg_batch<R, false><<<b.nblk, kSegAtoms, b.smem, s>>>(args, b.d_off, nrep);
}

cudaError_t launch_drift_batch(cudaStream_t s, bool fp64, bool ev, const BatchLaunch& b, int nrep) {
  if (b.nblk == 0) return cudaSuccess;
  if (fp64)
    launch_drift_batch_t<double>(s, ev, b, nrep);
  else
    launch_drift_batch_t<float>(s, ev, b, nrep);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t prepare_sum_batch_t(const std::vector<relres_ctx*>& cs, const std::vector<StepParams>& sp,
                                       double* const* d_vel, BatchLaunch* b) {
  std::vector<SumArgs<R>> args(cs.size());
  std::vector<int> off(cs.size() + 1, 0);
  for (size_t r = 0; r < cs.size(); ++r) {
    args[r] = sum_args<R>(cs[r], sp[r], d_vel[r]);
    off[r + 1] = off[r] + sum_blocks(cs[r]);
  }
  b->nblk = off.back();
  b->smem = b->smem_ev = 0;
  return upload_batch(b, args.data(), sizeof(SumArgs<R>) * args.size(), off);
}

cudaError_t prepare_sum_batch(const std::vector<relres_ctx*>& cs, const std::vector<StepParams>& sp,
                              double* const* d_vel, BatchLaunch* b) {
  return cs[0]->fp64 ? prepare_sum_batch_t<double>(cs, sp, d_vel, b) : prepare_sum_batch_t<float>(cs, sp, d_vel, b);
}

cudaError_t launch_sum_batch(cudaStream_t s, bool fp64, int k, const BatchLaunch& b, int nrep) {
  if (b.nblk == 0) return cudaSuccess;
  if (fp64)
    k_sum_batch<double><<<b.nblk, kThreads, 0, s>>>(static_cast<const SumArgs<double>*>(b.d_args), b.d_off, nrep, k);
  else
    k_sum_batch<float><<<b.nblk, kThreads, 0, s>>>(static_cast<const SumArgs<float>*>(b.d_args), b.d_off, nrep, k);
  return cudaGetLastError();
}

cudaError_t launch_write_back(relres_ctx* c, double* d_pos, double* d_vel, double dt) {
  (void)dt;
  const BoxConsts b = box_consts(c, 0.0);
  if (c->fp64)
    k_finish_md<double><<<grid_for(c->n), kThreads, 0, c->stream>>>(
        c->n, c->d_state, static_cast<const double*>(vel_state(c, d_vel)), static_cast<const double*>(c->d_f_tot),
        c->d_type, c->d_cdt, c->d_cdt_ff, c->d_xfx, b, d_vel, d_pos, c->d_pos_ret, nullptr);
  else
    k_finish_md<float><<<grid_for(c->n), kThreads, 0, c->stream>>>(
        c->n, c->d_state, static_cast<const float2*>(vel_state(c, d_vel)), static_cast<const float4*>(c->d_f_tot),
        c->d_type, c->d_cdt, c->d_cdt_ff, c->d_xfx, b, d_vel, d_pos, c->d_pos_ret, c->d_vel_ret);
  RELRES_LAUNCHED(c);
  return cudaGetLastError();
}

}  // namespace relres
