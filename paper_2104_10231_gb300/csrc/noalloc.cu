// relres_pair_forces_static: a RelRes pair evaluation that allocates nothing.
//
// Some callers cannot let a library allocate device memory: a host program
// that owns the whole GPU memory budget through its own allocator and loads
// this library as a plug-in, or a latency-critical loop in which cudaMalloc /
// cudaFree (which may synchronise the device) are not allowed.  For them this
// entry point evaluates the RelRes pair forces, energy and virial of a small
// system by an all-pairs FP64 sum, with every piece of scratch memory (the
// type-pair table and the per-block partial sums) in one file-scope static
// device array of fixed size.  The caller provides only inputs and outputs.
//
// Limits and sharing: at most RELRES_STATIC_MAX_ATOMS atoms and
// RELRES_MAX_TYPES types.  The array exists once per GPU that loads the
// library and stays allocated until the process exits.  All calls on a GPU
// share it: calls whose work overlaps on the GPU (different streams, or
// several host threads) race on it and must be serialised by the caller.
// Each call rewrites the table and every partial sum it reads, and clears the
// bad-type flag before its kernels run, so stale contents from an earlier
// call are never used.
//
// Atom types live on the device, so the host cannot check them: the kernel
// skips every pair whose type index is outside [0, n_types) (no table read
// with it), writes NaN forces for such an atom and raises a flag in the static
// array, and the reduction then writes NaN energy and virial.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress.
#include <atomic>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace relres {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticMaxBlocks = (RELRES_STATIC_MAX_ATOMS + kStaticThreads - 1) / kStaticThreads;
constexpr int kMaxDevices = 64;

struct StaticScratch {
  PairTab<double> tab[RELRES_MAX_TYPES * RELRES_MAX_TYPES];
  long long partial[kStaticMaxBlocks][kNQ];
  unsigned bad_type;  // set when an atom type was outside [0, n_types)
};

static __device__ __align__(256) StaticScratch g_static_scratch;

// host-side cache of the array's device address, per device (several host
// threads may look it up at once; each finds the same address)
static std::atomic<StaticScratch*> s_scratch_ptr[kMaxDevices];

__device__ __forceinline__ double poly5(const double* g, double d) {
  return (((g[4] * d + g[3]) * d + g[2]) * d + g[1]) * d + g[0];
}
__device__ __forceinline__ double poly4(const double* g, double d) {
  return ((g[3] * d + g[2]) * d + g[1]) * d + g[0];
}

// Eq. 20 as the sum of its FG and CG parts (see PairTab); returns -u'(r)/r
// in *fr and u(r) in *u.
__device__ __forceinline__ void relres_pair(const PairTab<double>& T, double r2, double* fr, double* u) {
  double f = 0.0, e = 0.0;
  if (r2 < T.rsp2) {  // FG part
    if (r2 < T.rsm2) {
      const double r2i = 1.0 / r2, r6i = r2i * r2i * r2i;
      f += r6i * (T.f12f * r6i - T.f6f) * r2i;
      e += r6i * (T.c12f * r6i - T.c6f) - T.e_fg_shift;
    } else {
      const double r = sqrt(r2), d = r - T.rsm;
      f += -poly4(T.fgd, d) / r;
      e += poly5(T.fg, d) - T.e_fg_shift;
    }
  }
  if (r2 < T.rcp2) {  // CG part (zero table entries for pairs without CG)
    if (r2 < T.rsm2) {
      e += T.e_cg_close;
    } else if (r2 < T.rsp2) {
      const double r = sqrt(r2), d = r - T.rsm, d2 = d * d;
      f += -(d2 * (T.ond4 * d + T.ond3)) / r;
      e += T.on0 + d2 * d * (T.on4 * d + T.on3) - T.gam_cm;
    } else if (r2 < T.rcm2) {
      const double r2i = 1.0 / r2, r6i = r2i * r2i * r2i;
      f += r6i * (T.f12c * r6i - T.f6c) * r2i;
      e += r6i * (T.c12c * r6i - T.c6c) - T.gam_cm;
    } else {
      const double r = sqrt(r2), d = r - T.rcm;
      f += -poly4(T.cgod, d) / r;
      e += poly5(T.cgo, d) - T.gam_cm;
    }
  }
  *fr = f;
  *u = e;
}

// One thread per atom, all partners j != i through shared-memory tiles.
__global__ void __launch_bounds__(kStaticThreads)
    k_allpairs_static(int n, int nt, const double* __restrict__ pos, const int* __restrict__ type,
                      double l0, double l1, double l2, const int* __restrict__ eoff,
                      const int* __restrict__ eidx, int with_excl, double* __restrict__ forces,
                      StaticScratch* scratch) {
  __shared__ double sx[kStaticThreads], sy[kStaticThreads], sz[kStaticThreads];
  __shared__ int stype[kStaticThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  double xi = 0.0, yi = 0.0, zi = 0.0;
  int ti = 0, e0 = 0, e1 = 0;
  bool bad_i = false;
  if (live) {
    xi = pos[3 * i];
    yi = pos[3 * i + 1];
    zi = pos[3 * i + 2];
    ti = type[i];
    bad_i = ti < 0 || ti >= nt;
    if (bad_i) {
      ti = 0;
      atomicOr(&scratch->bad_type, 1u);
    }
    if (with_excl) {
      e0 = eoff[i];
      e1 = eoff[i + 1];
    }
  }
  double fx = 0.0, fy = 0.0, fz = 0.0;
  double acc[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
  for (int base = 0; base < n; base += kStaticThreads) {
    const int jl = base + threadIdx.x;
    if (jl < n) {
      sx[threadIdx.x] = pos[3 * jl];
      sy[threadIdx.x] = pos[3 * jl + 1];
      sz[threadIdx.x] = pos[3 * jl + 2];
      stype[threadIdx.x] = type[jl];
    }
    __syncthreads();
    const int m = min(kStaticThreads, n - base);
    if (live) {
      for (int k = 0; k < m; ++k) {
        const int j = base + k;
        const int tj = stype[k];
        if (j == i || bad_i || tj < 0 || tj >= nt) continue;  // out-of-range types: no table read
        bool ex = false;
        for (int e = e0; e < e1; ++e) ex |= eidx[e] == j;
        if (ex) continue;
        double dx = xi - sx[k], dy = yi - sy[k], dz = zi - sz[k];
        dx -= l0 * rint(dx / l0);
        dy -= l1 * rint(dy / l1);
        dz -= l2 * rint(dz / l2);
        double fr, u;
        relres_pair(scratch->tab[ti * nt + tj], dx * dx + dy * dy + dz * dz, &fr, &u);
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        acc[0] += u;
        acc[1] += fr * dx * dx;
        acc[2] += fr * dy * dy;
        acc[3] += fr * dz * dz;
        acc[4] += fr * dx * dy;
        acc[5] += fr * dx * dz;
        acc[6] += fr * dy * dz;
      }
    }
    __syncthreads();
  }
  if (live) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    forces[3 * i] = bad_i ? nan : fx;
    forces[3 * i + 1] = bad_i ? nan : fy;
    forces[3 * i + 2] = bad_i ? nan : fz;
  }
  __shared__ double sh[(kStaticThreads / 32) * kNQ];
  block_sum<double, kNQ>(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < kNQ; ++q) scratch->partial[blockIdx.x][q] = to_fix_sum(0.5 * acc[q]);
}

__global__ void k_allpairs_static_reduce(int nblocks, const StaticScratch* scratch, double* energy,
                                         int with_energy, double* virial, int with_virial) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long tot[kNQ] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < kNQ; ++q) tot[q] += scratch->partial[b][q];
  const bool bad = scratch->bad_type != 0u;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  if (with_energy) energy[0] = bad ? nan : double(tot[0]) / kFix;
  if (with_virial)
    for (int q = 1; q < kNQ; ++q) virial[q - 1] = bad ? nan : double(tot[q]) / kFix;
}

}  // namespace
}  // namespace relres

using namespace relres;

extern "C" relres_status relres_pair_forces_static(const relres_params* p, int n_atoms, const int* d_type,
                                                   const double* d_pos, const double box[3],
                                                   const int* d_excl_offsets, const int* d_excl_index,
                                                   double* d_forces, double* d_energy, double* d_virial,
                                                   void* cuda_stream) {
  if (!p || !d_type || !d_pos || !box || !d_forces) return RELRES_ERR_ARG;
  if (n_atoms < 1 || n_atoms > RELRES_STATIC_MAX_ATOMS) return RELRES_ERR_ARG;
  if ((d_excl_offsets == nullptr) != (d_excl_index == nullptr)) return RELRES_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) return RELRES_ERR_ARG;
  // parameter preparation into stack buffers (no heap in this entry point's own code)
  double table[RELRES_MAX_TYPES * RELRES_MAX_TYPES * RELRES_PAIR_FIELDS];
  const relres_status ps = relres_prepare_table(p, table, int(sizeof(table) / sizeof(double)));
  if (ps != RELRES_OK) return ps;
  const int nt = p->n_types;
  double rmax = 0.0;
  PairTab<double> tabs[RELRES_MAX_TYPES * RELRES_MAX_TYPES];
  std::memset(tabs, 0, sizeof(tabs));
  for (int k = 0; k < nt * nt; ++k) {
    const double* o = table + k * RELRES_PAIR_FIELDS;
    PairTab<double>& t = tabs[k];
    const double s6f = std::pow(o[1], 6.0), s6c = std::pow(o[3], 6.0);
    t.c12f = 4.0 * o[0] * s6f * s6f;
    t.c6f = 4.0 * o[0] * s6f;
    t.f12f = 12.0 * t.c12f;
    t.f6f = 6.0 * t.c6f;
    t.rsm = o[4];
    t.rsm2 = o[4] * o[4];
    t.rsp2 = o[5] * o[5];
    for (int m = 0; m < 5; ++m) t.fg[m] = o[8 + m];
    for (int m = 1; m < 5; ++m) t.fgd[m - 1] = m * o[8 + m];
    const double ws = o[5] - o[4];
    t.e_fg_shift = (((o[12] * ws + o[11]) * ws + o[10]) * ws + o[9]) * ws + o[8];
    t.c12c = 4.0 * o[2] * s6c * s6c;
    t.c6c = 4.0 * o[2] * s6c;
    t.f12c = 12.0 * t.c12c;
    t.f6c = 6.0 * t.c6c;
    t.rcm = o[6];
    t.rcm2 = o[6] * o[6];
    t.rcp2 = o[7] * o[7];
    t.on0 = o[13];
    t.on3 = o[16];
    t.on4 = o[17];
    t.ond3 = 3.0 * o[16];
    t.ond4 = 4.0 * o[17];
    for (int m = 0; m < 5; ++m) t.cgo[m] = o[18 + m];
    for (int m = 1; m < 5; ++m) t.cgod[m - 1] = m * o[18 + m];
    t.gam_cm = o[23];
    t.e_cg_close = o[13] - o[23];
    rmax = std::fmax(rmax, std::fmax(o[5], o[2] > 0.0 ? o[7] : 0.0));
  }
  // minimum image needs every interaction range below half the box
  if (!(rmax < 0.5 * std::fmin(box[0], std::fmin(box[1], box[2])))) return RELRES_ERR_BOX;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RELRES_ERR_CUDA;
  StaticScratch* scratch = s_scratch_ptr[dev].load(std::memory_order_acquire);
  if (scratch == nullptr) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr) return RELRES_ERR_CUDA;
    scratch = static_cast<StaticScratch*>(ptr);
    s_scratch_ptr[dev].store(scratch, std::memory_order_release);
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // the table for this call (copied from the stack; a pageable-source copy
  // returns once the source has been read) and a cleared bad-type flag
  if (cudaMemcpyAsync(scratch->tab, tabs, sizeof(PairTab<double>) * nt * nt, cudaMemcpyHostToDevice,
                      stream) != cudaSuccess)
    return RELRES_ERR_CUDA;
  if (cudaMemsetAsync(&scratch->bad_type, 0, sizeof(unsigned), stream) != cudaSuccess) return RELRES_ERR_CUDA;
  int nblocks = (n_atoms + kStaticThreads - 1) / kStaticThreads;
  int with_excl = d_excl_offsets ? 1 : 0;
  // cudaLaunchKernel returns the status of this launch only: an earlier
  // error of unrelated work is neither reported as this call's nor cleared
  int n = n_atoms, ntt = nt;
  double l0 = box[0], l1 = box[1], l2 = box[2];
  const int* eoff = with_excl ? d_excl_offsets : d_type;
  const int* eidx = with_excl ? d_excl_index : d_type;
  void* args1[] = {&n, &ntt, const_cast<double**>(&d_pos), const_cast<int**>(&d_type), &l0, &l1, &l2,
                   const_cast<int**>(&eoff), const_cast<int**>(&eidx), &with_excl, &d_forces, &scratch};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_allpairs_static), dim3(nblocks), dim3(kStaticThreads),
                       args1, 0, stream) != cudaSuccess)
    return RELRES_ERR_CUDA;
  const StaticScratch* cscratch = scratch;
  double* e_out = d_energy ? d_energy : d_forces;
  double* w_out = d_virial ? d_virial : d_forces;
  int with_e = d_energy ? 1 : 0, with_w = d_virial ? 1 : 0;
  void* args2[] = {&nblocks, &cscratch, &e_out, &with_e, &w_out, &with_w};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_allpairs_static_reduce), dim3(1), dim3(1), args2, 0,
                       stream) != cudaSuccess)
    return RELRES_ERR_CUDA;
  return RELRES_OK;
}
