// Internal declarations of librelres (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/relres.h"

namespace relres {

// ------------------------------------------------------------------ tables

// FP64 per-type-pair quantities of Section 2 (exported by relres_prepare_table).
struct PairRecord {
  double eps_fg = 0, sig_fg = 0, eps_cg = 0, sig_cg = 0;
  double rsm = 0, rsp = 0, rcm = 0, rcp = 0;
  double g_fg_m[5] = {0, 0, 0, 0, 0};  // f_{s-}^{FG}  (Eq. 17)
  double g_cg_p[5] = {0, 0, 0, 0, 0};  // f_{s+}^{CG}  (Eq. 18)
  double g_cg_m[5] = {0, 0, 0, 0, 0};  // f_{c-}^{CG}  (Eq. 17)
  double gam_cm = 0, gam_sp = 0, gam_sm = 0;  // Eq. 19
};

// Kernel form of one type pair.  The pair kernels evaluate Eq. 20 split
// exactly into a part on the FG list and a part on the CG list:
//   FG part: u^FG(r) - f_{s-}(dr_s) for r < r_s-;  f_{s-}(r - r_s-) - f_{s-}(dr_s)
//            on [r_s-, r_s+);  0 beyond.
//   CG part: f_{s+}(0) - Gamma_{c-} for r < r_s-;  f_{s+}(r - r_s-) - Gamma_{c-} on
//            [r_s-, r_s+);  u^CG(r) - Gamma_{c-} on [r_s+, r_c-);
//            f_{c-}(r - r_c-) - Gamma_{c-} on [r_c-, r_c+);  0 beyond.
// The sum reproduces Gamma_{s+} and Gamma_{s-} of Eq. 19.  An odd number of
// 4-byte words per row keeps shared-memory rows on different banks.
template <typename R>
struct PairTab {
  R c12f, c6f, f12f, f6f;   // FG LJ: 4 eps sig^12, 4 eps sig^6, and x12 / x6
  R rsm, rsm2, rsp2;        // r_s-, r_s-^2, r_s+^2
  R fg[5];                  // f_{s-}^{FG} coefficients
  R fgd[4];                 // its derivative: g1, 2 g2, 3 g3, 4 g4
  R e_fg_shift;             // f_{s-}^{FG}(dr_s)
  R c12c, c6c, f12c, f6c;   // CG LJ
  R rcm, rcm2, rcp2;        // r_c-, r_c-^2, r_c+^2
  R on0, on3, on4, ond3, ond4;  // f_{s+}^{CG}: gamma_0, gamma_3, gamma_4, 3 gamma_3, 4 gamma_4
  R cgo[5];                 // f_{c-}^{CG}
  R cgod[4];                // its derivative
  R gam_cm;                 // Gamma_{c-}
  R e_cg_close;             // f_{s+}^{CG}(0) - Gamma_{c-}
  R pad;
};
static_assert(sizeof(PairTab<float>) % 8 == 4, "odd row length in words");

// Basis form of one type pair for the differentiable path.  Every smoothing
// coefficient (Eq. 17, Eq. 18) and shift (Eq. 19) is linear in the potential,
// so each part of Eq. 20 is C12 phi12(r) - C6 phi6(r), with phik the same
// construction applied to r^-k.  The rows hold, for k = 12 and 6: the FG
// switch-off polynomial and its shift f(dr_s), the CG switch-on and
// switch-off polynomials and Gamma_{c-}; and the current coefficients.
template <typename R>
struct BasisTab {
  R rsm, rsp, rcm, rcp;
  R fg[2][5], fg_sh[2];             // FG part: f_{s-}[r^-k], f_{s-}[r^-k](dr_s)  (k = 12, 6)
  R on[2][5], off[2][5], gam[2];    // CG part: f_{s+}[r^-k], f_{c-}[r^-k], Gamma_{c-}[r^-k]
  R c12f, c6f, c12c, c6c;           // 4 eps sig^12, 4 eps sig^6 (FG, CG)
};

std::string build_pair_records(const relres_params* p, std::vector<PairRecord>* out);
void build_basis_tables(const std::vector<PairRecord>& recs, int shift, std::vector<BasisTab<float>>* tf,
                        std::vector<BasisTab<double>>* td);
void build_kernel_tables(const std::vector<PairRecord>& recs, std::vector<PairTab<float>>* tf,
                         std::vector<PairTab<double>>* td);
void mix_pair(int mixing, double ea, double sa, double eb, double sb, double* e, double* s);
bool sum_rule(int nt, const double* eps, const double* sig, int mixing, const int* ci,
              const int* cj, double* eps_cg, double* sig_cg);

// ------------------------------------------------------------------ device state

enum : unsigned {
  F_REBUILD = 1u,       // an atom moved more than skin/2 since the last build
  F_OVERFLOW_FG = 2u,   // an FG list exceeded its capacity at the last build
  F_OVERFLOW_CG = 4u,
  F_NONFINITE = 8u,     // a non-finite force
  F_DIRTY = 16u,        // incoming positions differ from the cached state
  F_BADCELL = 32u,      // a computed cell index was out of range (access skipped)
  F_PRUNE = 64u,        // an atom moved more than delta/2 since the last pruning pass
  F_VDIRTY = 128u,      // incoming velocities differ from the ones returned last
};

struct DevState {
  unsigned flags;
  int max_fg, max_cg;
  int ev;                   // this step evaluates energy and virial
  double a, b;              // next drift: u <- a u + b (dt/2m) F
  float a_hi, a_lo, b_hi, b_lo;  // the same as float-float (FP32 path)
  double alpha;             // last thermostat factor
  unsigned long long step;  // global step counter (thermostat random stream)
  long long local_step;     // steps done in the current relres_step call
  long long n_builds;
  unsigned long long tot_fg, tot_cg;  // list entries at the last build
  unsigned long long n_prunes;        // pruning passes (each rebuild is followed by one)
  unsigned long long tot_in_fg, tot_in_cg;  // pruned-list entries summed over all passes
  int thermo_row;
  unsigned done_blocks;  // ticket counter of k_sum (zero between launches)
};

// Energy / virial partial sums are 64-bit fixed point (value * 2^32): exact,
// order-independent integer reductions.
constexpr double kFix = 4294967296.0;
constexpr int kNQ = 7;  // E, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz
// accumulator slots: FG pair sums, CG pair sums, kinetic energy, bonded energy
constexpr int kAccFg = 0, kAccCg = kNQ, kAccKe = 2 * kNQ, kAccEb = 2 * kNQ + 1, kNAcc = 2 * kNQ + 2;
constexpr int kBlockSteps = 100;  // steps between host status checks in relres_step
#ifndef RELRES_SEG_ATOMS
#define RELRES_SEG_ATOMS 256
#endif
constexpr int kSegAtoms = RELRES_SEG_ATOMS;  // atoms per segment (one block of the segment kernels)
// A segment record: atoms [a0, a1), then the bond, angle and dihedral ranges
// and the first atom of its prototype (a segment whose terms and incident-term
// lists are those of this one shifted by a0 - base; base = a0 where none).
constexpr int kSegRec = 9;
// exclusions as a per-atom bit mask over atom-id offsets -15 .. 15
constexpr int kExclMaskHalf = 15;
constexpr size_t kSegSmemMax = 48 * 1024;  // shared memory of a segment kernel (term slots + positions)
constexpr double kPruneDelta = 0.5;   // default margin of the pruned lists (Angstrom)
#define RELRES_ACC_DEFAULT RELRES_ACC_COMPENSATED
constexpr double kPruneSlack = 1e-3;  // added to the pruning radius: covers FP32 rounding of distances

// Launch configurations of the forces-only FP32 pair kernel: threads per slot
// (lanes that share one atom's list) and block size.  Index 0 is the default;
// the autotuner (relres_step, first call) times all of them.
struct PairConfig {
  int tpa, bs;
};
constexpr PairConfig kPairConfigs[] = {{1, 256}, {1, 128}, {1, 512}, {2, 256}, {4, 256}, {8, 256}, {2, 128}};
constexpr int kNPairConfigs = int(sizeof(kPairConfigs) / sizeof(kPairConfigs[0]));

struct Pos64 {  // FP64 mode sorted position: 64-bit fixed-point x, y, z and type
  long long x, y, z, t;
};

// Call-constant step parameters (kernel arguments).
struct StepParams {
  double dt;
  double t_target, tau, n_f, kt;  // CSVR
  double csvr_e;                  // exp(-dt / tau)
  unsigned long long seed;
  int thermo_every;
  double* thermo;  // device [rows][RELRES_THERMO_COLS] or null
};

// Cell grid of one list.  Full cells are at least one list radius wide (nf
// per axis).  With four or more of them on every axis each is cut into
// kXSplit slabs along x (xsplit), atoms are binned into those sub-cells, and
// the dense rank of a sub-cell is xsplit x the Morton rank of its full cell +
// its slab, so the atoms of a full cell are contiguous slots and the list
// build can give each atom the contiguous run of x-slabs within its list
// radius.
constexpr int kXSplit = 4;
struct Grid {
  int n[3];                  // binning cells per axis (x: nf[0] * xsplit)
  int nf[3];                 // full cells per axis
  int xsplit = 1;
  int ncell;                 // binning cells
  int ncell_full;
  int ntile;                 // tiles of the cell scan
  int* d_rank_of = nullptr;  // [n0*n1*n2] -> dense cell rank
  int* d_start = nullptr;    // [ncell+1]
  int* d_count = nullptr;    // [ncell] counts / cursors (zero between builds)
  int* d_tile = nullptr;     // [ntile] per-tile cell counts of the scan
};
constexpr int kScanTile = 4096;  // cells per block of the two-pass cell scan

// ------------------------------------------------------------------ context
}  // namespace relres

struct relres_ctx {
  // parameters
  relres_params prm{};
  std::vector<double> eps_fg, sig_fg;
  std::vector<int> is_hybrid;
  int n_types = 0;
  int hyb_mask = 0;
  bool has_cg = false;
  bool fp64 = false;
  std::vector<relres::PairRecord> recs;
  std::vector<relres::PairTab<float>> tab_f;
  std::vector<relres::PairTab<double>> tab_d;
  double rlist_fg_cut = 0, rlist_cg_cut = 0;  // max r_s+, max r_c+ over pairs
  cudaStream_t stream = nullptr;
  std::string err;

  // differentiable path: basis tables (BasisTab<float or double>[n_types^2]),
  // per-type-pair gradient totals, and lazily allocated gradient buffers
  std::vector<relres::BasisTab<float>> basis_f;
  std::vector<relres::BasisTab<double>> basis_d;
  void* d_basis = nullptr;
  double* d_gc = nullptr;     // [n_types^2][4]
  void* d_g_fg = nullptr;     // dL/dF in FG slot order
  void* d_g_cg = nullptr;     // dL/dF in CG slot order
  void* d_gx_fg = nullptr;    // dL/dx, FG part, caller order
  void* d_gx_cg = nullptr;    // dL/dx, CG part (hybrids), caller order
  double* d_zero_n3 = nullptr;
  int grad_n = 0;             // atoms the gradient buffers were allocated for

  // device tables
  void* d_tab = nullptr;  // PairTab<float or double>[n_types^2]
  void* d_tabd = nullptr; // PairTab<double>[n_types^2] (energies of the FP32 path)
  double* d_cdt = nullptr;   // per type: (dt/2m) * ftm2v  (set per step call)
  float2* d_cdt_ff = nullptr;  // the same as float-float (FP32 path)
  float* d_kec = nullptr;      // per type: m / 2 in kcal/mol per (A/fs)^2, FP32
  double* d_mass = nullptr;  // per type mass
  std::vector<double> h_cdt = std::vector<double>(RELRES_MAX_TYPES, 0.0);
  double consts_dt = 0.0;  // time step of the per-type constants on the device (0: none yet)

  // topology
  int n = 0, n_h = 0;
  bool have_topo = false;
  std::vector<int> h_type;
  std::vector<double> mass_by_type;
  int* d_type = nullptr;
  int* d_excl_off = nullptr;
  int excl_window = 0;  // max |i - j| over excluded pairs
  int* d_excl_idx = nullptr;
  // per atom i, bit (j - i + kExclMaskHalf) set for every excluded j and for
  // j = i; allocated only when excl_window <= kExclMaskHalf
  unsigned* d_excl_mask = nullptr;
  int n_bonds = 0, n_angles = 0, n_dih = 0;
  int4* d_bonds = nullptr;      // i, j, type, 0
  int4* d_angles = nullptr;     // i, vertex, k, type
  int4* d_dihs = nullptr;       // i, j, k, l
  int* d_dih_type = nullptr;
  double* d_bond_par = nullptr;   // k, r0 per type
  double* d_angle_par = nullptr;  // k, theta0 per type
  double* d_dih_par = nullptr;    // K1..K4 per type
  float* d_bond_fpar = nullptr;   // FP32 path: k, r0 hi, r0 lo, 0 per type
  float* d_angle_fpar = nullptr;  // FP32 path: k, theta0, cos hi/lo, sin hi/lo, 0, 0 per type
  int* d_inc_off = nullptr;   // incident terms per atom (CSR)
  int* d_inc = nullptr;       // (kind << 30) | (role << 28) | term
  long long* d_vir_dummy = nullptr;

  // box and grids
  bool have_box = false;
  double box[3] = {0, 0, 0};
  double skin_cg = 0;
  relres::Grid gfg, gcg;
  bool have_lists = false;

  // positions and sorting
  unsigned long long* d_xfx = nullptr;  // [n*3] 64-bit fixed point, caller order
  int4* d_ref = nullptr;                // [n] hi32 positions at the last build
  int4* d_ref_p = nullptr;              // [n] hi32 positions at the last pruning pass
  int* d_cell_fg = nullptr;
  int* d_cell_cg = nullptr;
  int* d_slot_fg = nullptr;             // arrival rank of the atom inside its cell
  int* d_slot_cg = nullptr;
  int* d_perm_fg = nullptr;             // FG slot -> atom
  int* d_rank_fg = nullptr;             // atom -> FG slot
  int* d_perm_cg = nullptr;             // CG slot -> atom
  int* d_rank_cg = nullptr;             // atom -> CG slot, -1 for ordinary
  int4* d_pos_fg = nullptr;             // [n] sorted hi32 positions + type
  int4* d_pos_cg = nullptr;             // [n_h]
  relres::Pos64* d_pos_fg64 = nullptr;  // FP64 mode
  relres::Pos64* d_pos_cg64 = nullptr;

  // lists
  int cap_fg = 0, cap_cg = 0;
  int* d_nbr_fg = nullptr;  // [cap_fg/4][n][4]: entry k of slot s at ((k/4)*n + s)*4 + k%4
  int* d_cnt_fg = nullptr;  // [n]
  int* d_nbr_cg = nullptr;  // [cap_cg][n_h]
  int* d_cnt_cg = nullptr;  // [n_h]
  int last_max_fg = 0, last_max_cg = 0;
  double last_mean_fg = 0, last_mean_cg = 0;
  // pruned lists (dynamic pruning): the entries of the lists above whose
  // distance was below the interaction cutoff + prune_delta at the last
  // pruning pass, same layout and capacity; the pair kernels walk these
  double prune_delta = relres::kPruneDelta;  // <= 0: no pruning (pair kernels walk the lists above)
  bool prune_on = false;                     // prune_delta > 0 and the inner lists are allocated
  int* d_nbr_fg_in = nullptr;
  int* d_cnt_fg_in = nullptr;
  int* d_nbr_cg_in = nullptr;
  int* d_cnt_cg_in = nullptr;

  // forces (caller order): float4 per atom (FP32) or double[3] per atom (FP64)
  void* d_f_fg = nullptr;
  void* d_f_cg = nullptr;
  void* d_f_tot = nullptr;
  void* d_f_bond = nullptr;  // bonded forces from the segmented drift kernel
  // FP32 path: the velocity state of relres_step (u, see md.cu) as float-float
  // pairs [3n] (the caller's FP64 velocities are read at the start of a call
  // and written at its end); the FP64 path keeps u in the caller's array
  float2* d_uff = nullptr;
  bool forces_valid = false;
  // what the last relres_step returned ([3n] positions, [3n] velocities) and
  // whether the state is still that call's end state (io_valid; io_dt its
  // time step): a call given those same arrays continues from that state
  // (FP32: the velocity state and the thermostat factors too) without
  // reading the arrays again
  double* d_pos_ret = nullptr;
  double* d_vel_ret = nullptr;
  bool io_valid = false;
  double io_dt = 0.0;

  // bonded-term force slots: bonds 2 per term, then angles 3, then dihedrals 4
  void* d_tf = nullptr;
  // segments of whole molecules for the fused bonded + force-sum kernel:
  // [n_seg][kSegRec] = atom range, the prototype's bond, angle and dihedral
  // ranges, the prototype's first atom
  int* d_seg = nullptr;
  int n_seg = 0, seg_slots = 0, n_seg_proto = 0;
  bool seg_ok = false;
  bool use_seg = true;  // the fused kernel where segments exist (relres_set_option)
  // force sum and drift as programmatic dependent launches (untimed steps)
  bool use_pdl = true;
  // reductions: 64-bit fixed-point accumulators (kNAcc), cleared by their reader
  long long* d_acc = nullptr;
  double* d_draws = nullptr;  // CSVR random numbers of the current block of steps, 2 per step
  relres::DevState* d_state = nullptr;
  unsigned* d_open = nullptr;  // device word that always reads F_REBUILD (un-gated launches)
  void* d_dummy = nullptr;     // valid target for pointer arguments a kernel does not use
  relres::DevState* h_state = nullptr;  // pinned mirror
  double* d_out_scratch = nullptr;      // [16]

  // rollback snapshot for relres_step
  unsigned long long* d_snap_x = nullptr;
  double* d_snap_v = nullptr;
  void* d_snap_f = nullptr;
  relres::DevState* d_snap_state = nullptr;

  long long n_builds = 0;
  long long n_steps = 0;
  unsigned long long step_counter = 0;

  // instrumentation
  long long n_launches = 0;
  bool timing = false;
  unsigned timing_mask = ~0u;  // timed classes (bit k: relres_timing_class k)
  int timing_every = 1;        // time only every timing_every-th step of a call
  int cur_step = 0;            // step of the call being recorded (0 outside relres_step)
  struct Mark {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Mark> marks;
  size_t ev_used = 0;

  // CUDA graph of one block of MD steps (relres_step): the list rebuild of
  // each step is a conditional node whose flag a one-thread kernel sets from
  // the device displacement trigger.  Everything below is baked into the
  // instantiated graph; it is re-captured when any of it changes.
  int pair_cfg = 0;        // index into kPairConfigs
  int force_acc = RELRES_ACC_DEFAULT;  // relres_accumulation of the FP32 pair kernels
  int tune_mode = -1;      // -1: autotune on the first relres_step; >= 0: fixed configuration
  bool tuned = false;
  bool use_graphs = true;
  long long buf_gen = 0;  // bumped whenever a buffer a graph may reference is reallocated
  struct StepGraph {
    bool valid = false;
    int blk = 0, ev_phase = 0, thermo_every = 0, timing = 0, pair_cfg = 0, t_every = 1, t_phase = 0;
    unsigned t_mask = 0;
    double dt = 0, t_target = 0, tau = 0, n_f = 0, kt = 0;
    unsigned long long seed = 0;
    const double* vel = nullptr;
    double* thermo = nullptr;
    long long gen = -1;
    cudaGraphExec_t exec = nullptr;
    std::vector<Mark> marks;          // event pairs recorded by the graph's own nodes
    std::vector<cudaEvent_t> events;  // owned by the graph
    long long k_parent = 0;           // kernels per launch outside the rebuild bodies
    long long k_body = 0;             // kernels per executed rebuild body
    long long k_prune = 0;            // kernels per executed pruning body (separate pruning pass)
    unsigned long long last_use = 0;  // cache recency
  };
  // Captured step graphs, one per block shape in use (a call of n steps runs
  // blocks of 100 and one shorter remainder, so a repeated call needs two);
  // the least recently used one is dropped when the cache is full.
  static constexpr int kMaxStepGraphs = 4;
  std::vector<StepGraph> sgs;
  int sg_cur = -1;                  // graph of the block being run
  unsigned long long sg_clock = 0;
  cudaStream_t cap_stream = nullptr;   // capture of the step graph
  cudaStream_t body_stream = nullptr;  // capture of the conditional rebuild bodies
  std::vector<Mark>* cap_marks = nullptr;     // non-null while capturing with timing
  std::vector<cudaEvent_t>* cap_events = nullptr;
  size_t cap_used = 0;
  double t_ms[RELRES_T_NCLASS] = {};
  long long t_cnt[RELRES_T_NCLASS] = {};
};

namespace relres {

// ------------------------------------------------------------------ launchers
// All launchers enqueue on ctx->stream and return cudaGetLastError().

// positions
cudaError_t launch_convert(relres_ctx* c, const double* d_pos);
cudaError_t launch_check_io(relres_ctx* c, const double* d_pos, const double* d_vel);
cudaError_t launch_write_back(relres_ctx* c, double* d_pos, double* d_vel, double dt);

// neighbour lists; gate: device flag word (rebuild only if F_REBUILD set) or null
cudaError_t launch_rebuild(relres_ctx* c, const unsigned* gate);
// sets the conditionals of a graph's rebuild node (F_REBUILD) and, with a
// separate pruning pass (with_prune), of its pruning node (F_REBUILD or
// F_PRUNE) from the device flag word
cudaError_t launch_decide(relres_ctx* c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle hp,
                          int with_prune);
cudaError_t launch_lists(relres_ctx* c, const unsigned* gate);
// pruning pass: inner lists from the full ones at the current positions
// (gate: runs if F_REBUILD or F_PRUNE is set)
cudaError_t launch_prune(relres_ctx* c, const unsigned* gate);

// Forces.  ev: this evaluation also adds energies and virial to the
// accumulators (d_acc).  The pair kernel covers both lists in one launch
// (which: 1 = FG list only, 2 = CG list only, 3 = both).  launch_finish runs
// the bonded-term kernel and the per-atom force sum; with d_vel it also adds
// the kinetic energy of u + c F.
// With pruning on and one thread per slot, a launch that finds F_REBUILD or
// F_PRUNE set walks the full lists and writes the pruned ones as it goes.
cudaError_t launch_pairs(relres_ctx* c, bool ev, int which = 3);
// whether this context's pair launches prune (pruning on, one thread per
// slot); otherwise a separate pruning pass precedes them when it is due
bool pairs_prune(const relres_ctx* c);
cudaError_t launch_finish(relres_ctx* c, bool ev, double* d_forces_out, const double* d_vel);
cudaError_t launch_reduce_out(relres_ctx* c, double* d_energy, double* d_virial);
// backward pass of the pair interaction (grad.cu): per-type-pair totals into
// d_gc, dL/dx (FP64, caller order) into d_grad_pos if non-null
cudaError_t launch_pair_grad(relres_ctx* c, const double* d_grad_forces, double g_energy, double* d_grad_pos);

// MD
cudaError_t upload_type_consts(relres_ctx* c, double dt);
// drift of one step; where the atoms form segments of whole molecules it also
// evaluates the bonded forces of the new positions (d_f_bond; energy if ev)
// after_sum: the previous kernel of the stream is the force sum of the
// previous step (the drift may then be a programmatic dependent launch)
cudaError_t launch_drift(relres_ctx* c, const StepParams& sp, double* d_vel, bool ev, bool after_sum);
// after the pair kernel: total forces, kinetic energy, thermostat and step
// bookkeeping (k_sum with the thermostat in its last block, or the
// finish + k_thermo pair where there are no segments)
cudaError_t launch_end_of_step(relres_ctx* c, const StepParams& sp, int k, bool ev, double* d_vel);
cudaError_t launch_csvr_draws(relres_ctx* c, const StepParams& sp, int count);
cudaError_t launch_thermo(relres_ctx* c, const StepParams& sp, int k);
cudaError_t launch_call_start(relres_ctx* c, bool reset_ab);
// FP32 path: caller's velocities -> the float-float state (start of a call)
cudaError_t launch_vel_in(relres_ctx* c, const double* d_vel);
// the velocity state of a call: the float-float array (FP32) or the caller's (FP64)
inline void* vel_state(relres_ctx* c, double* d_vel) {
  return c->fp64 ? static_cast<void*>(d_vel) : static_cast<void*>(c->d_uff);
}
cudaError_t launch_flags_and(relres_ctx* c, unsigned keep);

// ---- batched launches (relres_batch_step): one launch of a kernel class
// covers every replica.  d_args holds one argument struct per replica and
// d_off the cumulative block counts (block b works for the replica r with
// d_off[r] <= b < d_off[r + 1]); both are uploaded before the step graph is
// captured and stay valid while the replicas' buffers do.
struct BatchLaunch {
  void* d_args = nullptr;
  int* d_off = nullptr;
  size_t args_bytes = 0;
  int n_off = 0;
  int nblk = 0;
  size_t smem = 0, smem_ev = 0;
};
// (re)allocates the device tables of b as needed and copies args and off in (synchronous)
cudaError_t upload_batch(BatchLaunch* b, const void* args, size_t bytes, const std::vector<int>& off);
void free_batch(BatchLaunch* b);
cudaError_t prepare_pairs_batch(const std::vector<relres_ctx*>& cs, BatchLaunch* b);
cudaError_t launch_pairs_batch(cudaStream_t s, bool fp64, int acc, bool ev, const BatchLaunch& b, int nrep);
cudaError_t prepare_drift_batch(const std::vector<relres_ctx*>& cs, const std::vector<StepParams>& sp,
                                double* const* d_vel, BatchLaunch* b);
cudaError_t launch_drift_batch(cudaStream_t s, bool fp64, bool ev, const BatchLaunch& b, int nrep);
cudaError_t prepare_sum_batch(const std::vector<relres_ctx*>& cs, const std::vector<StepParams>& sp,
                              double* const* d_vel, BatchLaunch* b);
cudaError_t launch_sum_batch(cudaStream_t s, bool fp64, int k, const BatchLaunch& b, int nrep);
// the list rebuild of every replica whose displacement trigger fired (d_states[r]->flags & F_REBUILD):
// a work-list kernel and seven batched rebuild kernels (neighbor.cu)
struct RebuildBatch {
  BatchLaunch args;  // BuildArgs per replica
  BatchLaunch nbt;   // blocks of each kernel class per replica
  int* d_wl = nullptr;  // work list written on the device each step
  size_t wl_ints = 0;
};
cudaError_t prepare_rebuild_batch(const std::vector<relres_ctx*>& cs, RebuildBatch* rb);
// the work list of this step; sets `any` (a graph conditional) iff some replica rebuilds
cudaError_t launch_worklist(cudaStream_t s, const RebuildBatch& rb, DevState* const* d_states, int nrep,
                            cudaGraphConditionalHandle any);
// the seven batched rebuild kernels over the work list
cudaError_t launch_rebuild_batch(cudaStream_t s, const RebuildBatch& rb, int nrep);
void free_rebuild_batch(RebuildBatch* rb);
// kernels of one list rebuild: k_bin, k_scan_tiles, k_scan_add, k_scatter,
// k_sort_cells, k_pack, k_list
constexpr long long kRebuildKernels = 7;

// MD steps take the segmented drift + bonded kernel and k_sum
inline bool step_segments(const relres_ctx* c) { return c->seg_ok && c->use_seg; }

// FP64 forces-only pair launches: 32-thread blocks for a system with fewer
// 256-slot blocks than SMs, else 256; eight threads per slot (walk_ordered)
// for one whose slots fill fewer than four warps per SM with one thread each
constexpr int kPartSMs = 152;
constexpr int kFp64SmallTpa = 8;
inline int fp64_pair_block(const relres_ctx* c) { return (c->n + 255) / 256 < kPartSMs ? 32 : 256; }
inline int fp64_pair_tpa(const relres_ctx* c) {
  const long long slots = (long long)c->n + ((c->has_cg && c->n_h > 0) ? c->n_h : 0);
  return slots < 4LL * 32 * kPartSMs ? kFp64SmallTpa : 1;
}

// the lists the pair kernels walk: the pruned ones when pruning is on
inline const int* walk_nbr_fg(const relres_ctx* c) { return c->prune_on ? c->d_nbr_fg_in : c->d_nbr_fg; }
inline const int* walk_cnt_fg(const relres_ctx* c) { return c->prune_on ? c->d_cnt_fg_in : c->d_cnt_fg; }
inline const int* walk_nbr_cg(const relres_ctx* c) { return c->prune_on ? c->d_nbr_cg_in : c->d_nbr_cg; }
inline const int* walk_cnt_cg(const relres_ctx* c) { return c->prune_on ? c->d_cnt_cg_in : c->d_cnt_cg; }

}  // namespace relres
