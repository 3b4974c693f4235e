// Device helpers shared by the librelres kernels.
#pragma once

#include <cuda_runtime.h>

#include "relres_internal.h"

// Every launcher counts its kernels.  Building with -DRELRES_DEBUG_SYNC also
// synchronises after each launch and reports the first failing kernel site.
#ifdef RELRES_DEBUG_SYNC
#include <cstdio>
#define RELRES_LAUNCHED(c)                                                                   \
  do {                                                                                       \
    ++(c)->n_launches;                                                                       \
    const cudaError_t e_ = cudaDeviceSynchronize();                                          \
    if (e_ != cudaSuccess) std::fprintf(stderr, "relres: %s:%d %s\n", __FILE__, __LINE__,    \
                                        cudaGetErrorString(e_));                             \
  } while (0)
#else
#define RELRES_LAUNCHED(c) (++(c)->n_launches)
#endif

namespace relres {

constexpr int kThreads = 256;

// Programmatic dependent launch: a kernel launched with the
// programmatic-stream-serialization attribute may start before the previous
// kernel of its stream has finished.  grid_dependency_wait() blocks until that
// kernel has finished and its memory is visible (it returns at once for a
// kernel launched the ordinary way); grid_dependents_launch() lets the next
// such kernel start once every block of this grid has called it or exited.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Positions are periodic 64-bit fixed point: u = frac(x / L) * 2^64.  Integer
// differences wrap modulo 2^64, which is exactly the minimum image of an
// orthorhombic box, and the upper 32 bits give the 32-bit form the FP32 pair
// kernels read (resolution L / 2^32, 8e-8 A for L = 345 A).
__device__ __forceinline__ unsigned long long to_fixed(double x, double inv_l) {
  double s = x * inv_l;
  s -= floor(s);
  if (!(s < 1.0)) s = 0.0;
  return __double2ull_rz(s * 18446744073709551616.0);
}

__device__ __forceinline__ double from_fixed(unsigned long long u, double l_2m64) {
  return __ull2double_rn(u) * l_2m64;
}

__device__ __forceinline__ int hi32(unsigned long long u) { return int(unsigned(u >> 32)); }

// wrapped difference a - b of 32-bit periodic coordinates
__device__ __forceinline__ float dfix32(int a, int b, float scale) {
  return float(int(unsigned(a) - unsigned(b))) * scale;
}

__device__ __forceinline__ double dfix64(long long a, long long b, double scale) {
  return __ll2double_rn((long long)((unsigned long long)a - (unsigned long long)b)) * scale;
}

// cell coordinate of a 32-bit periodic coordinate on an n-cell axis:
// floor(frac * n) = high word of the 32 x 32 bit product
__device__ __forceinline__ int cell_of(int h, int n) { return int(__umulhi(unsigned(h), unsigned(n))); }

// No kernel ever receives a null pointer: optional buffers come with an int
// flag and a valid (possibly unused) pointer.  `gate` points at the device flag
// word of a step (rebuild only when F_REBUILD is set; pruning when F_REBUILD
// or F_PRUNE is set) or at a word that always has F_REBUILD set.
// Replica of block b in a batched launch: the r with off[r] <= b < off[r + 1]
// (off: cumulative block counts of the nrep replicas, off[0] = 0).
__device__ __forceinline__ int batch_replica(const int* __restrict__ off, int nrep, int b) {
  int lo = 0, hi = nrep - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool gate_closed(const unsigned* gate, unsigned mask = F_REBUILD) {
  return (*(volatile const unsigned*)gate & mask) == 0u;
}

// Pruning: append entry j to a slot's pruned list (chunked layout, slot
// pointer out4 = list + slot as int4, k entries so far) if kept.  buf is a
// shift register of the last four kept entries (oldest in x): once k reaches a
// multiple of four it holds the chunk just completed, which is written as one
// 16-byte store.  No branch depends on keep.
__device__ __forceinline__ void keep_entry(bool keep, int j, int& k, int4& buf, int4* out4, int nslots) {
  buf.x = keep ? buf.y : buf.x;
  buf.y = keep ? buf.z : buf.y;
  buf.z = keep ? buf.w : buf.z;
  buf.w = keep ? j : buf.w;
  k += keep ? 1 : 0;
  if (keep && (k & 3) == 0) out4[size_t((k >> 2) - 1) * nslots] = buf;
}
// The last, partial chunk (k % 4 entries, the newest in buf.w).
__device__ __forceinline__ void keep_tail(int k, const int4& buf, int4* out4, int nslots) {
  const int r = k & 3;
  if (r == 0) return;
  const int4 t = r == 1 ? make_int4(buf.w, buf.w, buf.w, buf.w)
                        : (r == 2 ? make_int4(buf.z, buf.w, buf.w, buf.w) : make_int4(buf.y, buf.z, buf.w, buf.w));
  out4[size_t(k >> 2) * nslots] = t;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of NV values per thread; result valid in thread 0.
// `sh` must hold (blockDim.x / 32) * NV elements.
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid * NV + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      T s = T(0);
      for (int w = 0; w < nw; ++w) s += sh[w * NV + q];
      v[q] = s;
    }
  }
}

__device__ __forceinline__ long long to_fix_sum(double v) { return __double2ll_rn(v * kFix); }

// ---- float-float ("double-single") arithmetic (Dekker 1971; Knuth's
// two-sum) for the FP32 path where FP32 alone is not enough: stiff bonds and
// the pair energies of energy steps.  A value is hi + lo with |lo| <=
// ulp(hi)/2.  The rounding intrinsics keep the error-free transformations
// from being contracted into FMAs.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff ff_quick(float a, float b) {  // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff t = ff_two_sum(a.hi, b.hi);
  return ff_quick(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = fmaf(a.hi, b.hi, -p);
  return ff_quick(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi))));
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.f)) return ff{0.f, 0.f};
  const float r = sqrtf(a.hi);
  const float p = __fmul_rn(r, r);
  const float pe = fmaf(r, r, -p);
  return ff_quick(r, __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo), __fmul_rn(2.f, r)));
}
__device__ __forceinline__ float ff_val(ff a) { return __fadd_rn(a.hi, a.lo); }
// float-float times float
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = fmaf(a.hi, b, -p);
  return ff_quick(p, __fadd_rn(e, __fmul_rn(a.lo, b)));
}
// float -> int64 rounded to nearest (ties to even), for |v| < 2^54, with
// 32-bit conversions only (conversions to and from 64-bit integers run at the
// FP64 rate on this part).  v = k 2^24 + rem: k = rint(v / 2^24) has at most
// 24 significant bits (so float(k) and k 2^24 are exact) and rem = v - k 2^24
// is exact with |rem| <= 2^23.
__device__ __forceinline__ long long f2ll_rn(float v) {
  const int k = __float2int_rn(__fmul_rn(v, 5.9604644775390625e-8f));
  const float rem = __fsub_rn(v, __fmul_rn(__int2float_rn(k), 16777216.f));
  return (long long)k * 16777216ll + (long long)__float2int_rn(rem);
}
// int64 -> float-float (~48 significant bits) from three 21-bit pieces, each
// converted exactly by a 32-bit conversion, summed with error-free additions
__device__ __forceinline__ ff ff_from_ll(long long d) {
  const float f1 = __fmul_rn(__int2float_rn(int(d >> 42)), 4398046511104.f);
  const float f2 = __fmul_rn(__int2float_rn(int((d >> 21) & 0x1fffffll)), 2097152.f);
  const float f3 = __int2float_rn(int(d & 0x1fffffll));
  const ff s = ff_two_sum(f1, f2);
  const ff u = ff_two_sum(s.hi, f3);
  return ff_quick(u.hi, __fadd_rn(u.lo, s.lo));
}
// float-float -> int64 (both parts rounded separately)
__device__ __forceinline__ long long ff2ll(ff v) { return f2ll_rn(v.hi) + f2ll_rn(v.lo); }
__device__ __forceinline__ ff ff_from(float a) { return ff{a, 0.f}; }
// 1/a: FP32 estimate and one Newton step in float-float
__device__ __forceinline__ ff ff_rcp(ff a) {
  const float y = __frcp_rn(a.hi);
  const ff e = ff_sub(ff_from(1.f), ff_mul(a, ff_from(y)));
  return ff_add(ff_from(y), ff_mul(ff_from(y), e));
}
// exact wrapped 32-bit fixed-point difference a - b, times the box scale s
__device__ __forceinline__ ff ff_fixed_diff32(int a, int b, ff s) {
  const int d = int(unsigned(a) - unsigned(b));
  const float hi = __int2float_rn(d);
  const float lo = __int2float_rn(d - __float2int_rn(hi));
  return ff_mul(ff_quick(hi, lo), s);
}

// Integer accumulators: a block's FP64 sum is converted to 64-bit fixed point
// and added with an integer atomic (exact, independent of order).
__device__ __forceinline__ void acc_add(long long* acc, double v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)to_fix_sum(v));
}

// 1/x in FP32: the hardware estimate (rcp.approx, about one ulp) refined by
// one Newton-Raphson step y + y (1 - x y), which leaves about one ulp as well.
// The correctly rounded __frcp_rn costs several more instructions plus a
// special-case branch; in the pair kernel's LJ core that was 12 % of the
// forces-only launch time.  Results below the smallest normal float are
// flushed to 0 (the pair kernel's padding distance, 3e38, gives 0).
// relres_eval_recip evaluates these functions for the tests.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_nr(float x) {
  const float y = rcp_approx(x);
  return fmaf(y, fmaf(-x, y, 1.f), y);
}

// FP64 1/x and 1/sqrt(x) from the FP32 hardware estimate plus one Newton
// step (relative error ~1e-13; FP64 division and square root are many times
// slower on this part).
__device__ __forceinline__ double rcp_d(double x) {
  const double y = double(rcp_approx(float(x)));
  return y * fma(-x, y, 2.0);
}
__device__ __forceinline__ double rsqrt_d(double x) {
  const double y = double(rsqrtf(float(x)));
  return y * fma(-0.5 * x * y, y, 1.5);
}

}  // namespace relres
