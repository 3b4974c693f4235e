/*
 * relres.h -- C ABI of librelres: GB300 (sm_103a) Relative Resolution
 * Lennard-Jones molecular dynamics.
 *
 * Method: M. Chaimovich & A. Chaimovich, "Relative Resolution: A
 * Computationally Efficient Implementation in LAMMPS", arXiv:2104.10231.
 * Near atom pairs interact through fine-grained (FG) LJ, switched off over
 * [r_s-, r_s+); pairs of hybrid sites (one per group of atoms) also interact
 * through coarse-grained (CG) LJ, switched on over the same shell and off over
 * [r_c-, r_c+).  The pair potential is Eq. 20 (Section 2.5), with the CG
 * parameters of Eq. 13 (Section 2.3), the smoothing polynomials of Eq. 16-18
 * (Section 2.4) and the shifts of Eq. 19.
 *
 * Conventions for every entry point
 *  - Units: kcal/mol, Angstrom, fs, g/mol, K ("real" units).
 *  - Pointers named d_* are CUDA device pointers owned by the caller; all
 *    other pointers are host pointers, read during the call only (the context
 *    copies what it keeps).  Positions and forces are row-major n_atoms x 3
 *    doubles (x0 y0 z0 x1 ...), in the caller's atom order.
 *  - Work is enqueued on the CUDA stream given to relres_create; calls return
 *    after it is enqueued unless stated otherwise.  Calls that must inspect a
 *    device status word (list overflow, rebuild, non-finite) synchronise that
 *    stream.
 *  - No call throws, traps or aborts.  Every call returns a relres_status;
 *    relres_last_error() gives a message for the last failure of a context.
 *  - A context is thread-compatible, not thread-safe: one host thread at a
 *    time per context.
 */
#ifndef RELRES_H
#define RELRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RELRES_MAX_TYPES 8
#define RELRES_THERMO_COLS 10 /* E_fg E_cg E_bonded KE Wxx Wyy Wzz Wxy Wxz Wyz */
#define RELRES_PAIR_FIELDS 26 /* see relres_prepare_table */

typedef enum relres_status {
  RELRES_OK = 0,
  RELRES_ERR_ARG = 1,           /* invalid argument: sizes, NULL, radii order, eps/sigma range */
  RELRES_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  RELRES_ERR_BOX = 3,           /* a cutoff does not fit the box (needs r_c+ < L/2 per axis) */
  RELRES_ERR_LIST_OVERFLOW = 4, /* neighbour list still too small after automatic regrowth */
  RELRES_ERR_NONFINITE = 5,     /* a non-finite position, force or energy */
  RELRES_ERR_STATE = 6,         /* call order: e.g. compute before topology / neighbours */
  RELRES_ERR_NOMEM = 7          /* device or host allocation failed */
} relres_status;

enum relres_mixing { RELRES_MIX_GEOMETRIC = 0, RELRES_MIX_LB = 1 };

/* RELRES_PREC_FP64: every pair and bonded term in FP64 (small systems).
 * RELRES_PREC_FP32: pair terms in FP32 from exact fixed-point coordinate
 * differences; per-atom sums in FP32; energy/virial totals, velocities and
 * positions in FP64 (64-bit fixed point for positions inside relres_step). */
enum relres_precision { RELRES_PREC_FP64 = 0, RELRES_PREC_FP32 = 1 };

/* How the FP32 pair kernels sum one atom's pair forces (relres_set_force_accumulation):
 * RELRES_ACC_FP32         FP32 running sums;
 * RELRES_ACC_COMPENSATED  float-float running sums (every term added with an
 *                         error-free two-sum: ~48-bit sums in FP32 arithmetic);
 * RELRES_ACC_FP64         FP64 running sums (each FP32 pair term converted and
 *                         added in FP64).
 * The sum is rounded to FP32 once, when the force is stored. */
enum relres_accumulation { RELRES_ACC_FP32 = 0, RELRES_ACC_COMPENSATED = 1, RELRES_ACC_FP64 = 2 };

typedef struct relres_ctx relres_ctx;

/*
 * Pair-style parameters (the pair_style / pair_coeff / pair_modify data of
 * Section 2.5).
 *   n_types        1..RELRES_MAX_TYPES atom types.
 *   eps_fg, sig_fg [n_types] FG LJ parameters per type (Eq. 11); eps >= 0,
 *                  sig > 0.
 *   is_hybrid      [n_types] 1 if sites of this type are hybrid (carry the CG
 *                  interaction of their group, Section 2.1), else 0.
 *   mixing         FG cross terms: geometric (eps, sig geometric means, Section
 *                  2.3) or Lorentz-Berthelot (sig arithmetic mean).
 *   eps_cg, sig_cg [n_types*n_types] explicit CG pair parameters (row-major
 *                  a*n_types+b), or NULL to derive them with Eq. 13.  Pairs
 *                  with an ordinary type must have eps_cg == 0 (Eq. 14);
 *                  otherwise RELRES_ERR_ARG.
 *   group_comp     [n_types*n_types] used when eps_cg == NULL: row a lists how
 *                  many FG sites of each type make up the group whose hybrid
 *                  site has type a (the hybrid site included).  Eq. 13 then
 *                  gives eps^CG and sig^CG of every hybrid type pair.  Rows of
 *                  ordinary types are ignored.
 *   r_si r_so r_ci r_co   the global radii r_s- <= r_s+ <= r_c- <= r_c+ (>0).
 *                  r- == r+ removes a smoothing zone.
 *   radii_pair     [n_types*n_types*4] per-pair override of the four radii
 *                  (symmetric), or NULL.
 *   shift          1: Eq. 19 in full (Gamma_{c-} = f_{c-}^{CG}(dr_c)); 0: the
 *                  "pair_modify shift no" of Section 2.5, Gamma_{c-} = 0 (and
 *                  Gamma_{s+}, Gamma_{s-} formed from Eq. 19 with that zero).
 *   skin           Verlet-list skin (Angstrom, >= 0); lists are rebuilt when
 *                  an atom has moved more than skin/2 since the last build.
 *   precision      RELRES_PREC_FP64 or RELRES_PREC_FP32.
 */
typedef struct relres_params {
  int n_types;
  const double* eps_fg;
  const double* sig_fg;
  const int* is_hybrid;
  int mixing;
  const double* eps_cg;
  const double* sig_cg;
  const int* group_comp;
  double r_si, r_so, r_ci, r_co;
  const double* radii_pair;
  int shift;
  double skin;
  int precision;
} relres_params;

/*
 * Molecular topology (host arrays, copied).
 *   type            [n_atoms] 0..n_types-1.
 *   mass_by_type    [n_types] g/mol, > 0.
 *   excl_offsets    [n_atoms+1], excl_index [excl_offsets[n_atoms]]: CSR lists
 *                   of the partners of each atom whose pair interaction is
 *                   removed (1-2, 1-3, ... as the force field wants); must be
 *                   symmetric.  Both NULL: no exclusions.  Applied to the FG
 *                   and the CG part alike.
 *   bonds           [2*n_bonds] atom pairs, bond_type [n_bonds] into
 *                   bond_k/bond_r0 [n_bond_types]: E = K (r - r0)^2.
 *   angles          [3*n_angles] (i, vertex, k), angle_type into angle_k /
 *                   angle_theta0 (radians): E = K (theta - theta0)^2.
 *   dihedrals       [4*n_dihedrals], dihedral_type into dihedral_k
 *                   [4*n_dihedral_types] = K1..K4 of the OPLS form
 *                   E = 1/2 [K1(1+cos p) + K2(1-cos 2p) + K3(1+cos 3p) + K4(1-cos 4p)].
 * Counts may be 0 with NULL arrays.
 */
typedef struct relres_topology {
  int n_atoms;
  const int* type;
  const double* mass_by_type;
  const int* excl_offsets;
  const int* excl_index;
  int n_bonds;
  const int* bonds;
  const int* bond_type;
  int n_bond_types;
  const double* bond_k;
  const double* bond_r0;
  int n_angles;
  const int* angles;
  const int* angle_type;
  int n_angle_types;
  const double* angle_k;
  const double* angle_theta0;
  int n_dihedrals;
  const int* dihedrals;
  const int* dihedral_type;
  int n_dihedral_types;
  const double* dihedral_k;
} relres_topology;

typedef struct relres_stats {
  int n_atoms, n_hybrid;
  int cap_fg, cap_cg;            /* list slots per atom / per hybrid */
  int max_fg, max_cg;            /* longest list at the last build */
  double mean_fg, mean_cg;       /* mean list length at the last build */
  double list_radius_fg;         /* max r_s+ + skin */
  double list_radius_cg;         /* max r_c+ + skin_cg (0 without CG pairs) */
  double skin_cg;                /* CG skin after clamping to L/2 - r_c+ */
  int grid_fg[3], grid_cg[3];    /* cells per axis */
  long long n_builds;            /* list builds since create */
  long long n_steps;             /* MD steps since create (also the thermostat counter) */
  int has_cg;                    /* 1 if any hybrid pair has eps^CG > 0 */
  long long n_launches;          /* CUDA kernels this context has launched */
  int pair_tpa, pair_block;      /* forces-only pair kernel: threads per atom, block size */
  double prune_delta;            /* pruning margin in Angstrom (0: pruning off) */
  long long n_prunes;            /* pruning passes since create (each build is followed by one) */
  double mean_fg_pruned, mean_cg_pruned;  /* mean pruned list length over all passes */
  int step_segments;             /* 1: MD steps evaluate bonded terms per segment of whole molecules
                                    inside the drift kernel; 0: separate bonded-term kernel */
  int force_acc;                 /* relres_accumulation of the FP32 pair kernels */
  int n_segments;                /* segments of whole molecules (0: no segmentation) */
  int n_segment_protos;          /* distinct segments: the others read the term records of an
                                    identical earlier one, shifted to their own atoms */
} relres_stats;

/* Kernel classes of relres_get_timings. */
enum relres_timing_class {
  RELRES_T_DRIFT = 0,    /* kick + drift + sorted scatter + rebuild trigger */
  RELRES_T_REBUILD = 1,  /* binning, scan, scatter, in-cell sort, pack */
  RELRES_T_LISTS = 2,    /* FG and CG Verlet lists */
  RELRES_T_PAIR = 3,     /* RelRes pair kernel over the FG and CG lists (one launch), forces only */
  RELRES_T_FINISH = 4,   /* force sum + bonded terms + kinetic energy */
  RELRES_T_THERMO = 5,   /* reductions + CSVR factor */
  RELRES_T_PAIR_EV = 6,  /* pair kernel on energy steps (forces + energy + virial) */
  RELRES_T_PRUNE = 7,    /* pruning pass of both lists (relres_set_prune) */
  RELRES_T_NCLASS = 8
};

/*
 * Host-only (no GPU needed): validate p and fill out[n_types*n_types*26]
 * with the per-pair quantities of Section 2, in FP64, pair a*n_types+b:
 *   eps_fg sig_fg eps_cg sig_cg r_s- r_s+ r_c- r_c+,
 *   gamma_{m-}^{FG} m=0..4 (Eq. 17 at r_s-), gamma_{m+}^{CG} (Eq. 18 at r_s+,
 *   gamma_4 with the sign that satisfies Eq. 8), gamma_{m-}^{CG} (Eq. 17 at
 *   r_c-), Gamma_{c-} Gamma_{s+} Gamma_{s-} (Eq. 19).
 * out_len is the capacity in doubles.  Errors: RELRES_ERR_ARG.
 */
relres_status relres_prepare_table(const relres_params* p, double* out, int out_len);

/*
 * Host-only: CG pair parameters of Eq. 13 for two groups given by FG site
 * compositions comp_i/comp_j [n_types] over per-type eps/sig with the given
 * mixing rule.  Writes *eps_cg, *sig_cg.  Errors: RELRES_ERR_ARG.
 */
relres_status relres_cg_params(int n_types, const double* eps_fg, const double* sig_fg,
                               int mixing, const int* comp_i, const int* comp_j,
                               double* eps_cg, double* sig_cg);

/*
 * Host-only: the chain rule through Eq. 13 when the CG parameters follow the
 * FG ones (p->group_comp gives the group compositions; the Eq. 13 CG
 * parameters of every hybrid type pair a, b are functions of p->eps_fg,
 * p->sig_fg and p->mixing).  Given the gradients of some scalar with respect
 * to the CG parameters of every type pair, g_eps_cg, g_sig_cg
 * [n_types*n_types] row-major (as relres_backward returns them), ADDS their
 * contribution to the gradients with respect to the per-type FG parameters,
 * g_eps_fg, g_sig_fg [n_types] (which the caller holds, e.g. initialised with
 * relres_backward's direct FG gradients):
 *   g_eps_fg[t] += sum_{a,b hybrid} g_eps_cg[ab] d eps^CG_ab / d eps_t
 *                                  + g_sig_cg[ab] d sig^CG_ab / d eps_t,
 * and likewise for sig_t.  Entries of pairs with an ordinary type are
 * ignored (Eq. 14: no CG term).  The eps derivative of a mixed pair
 * eps_{mu nu} = sqrt(eps_mu eps_nu) is taken as zero where eps_mu or eps_nu
 * is zero; Eq. 13 parameters that come out zero contribute nothing.
 * p->eps_cg must be NULL (the parameters follow Eq. 13).  Errors:
 * RELRES_ERR_ARG (invalid p as relres_prepare_table, NULL arrays, no
 * group_comp, explicit eps_cg, a non-finite gradient).
 */
relres_status relres_chain_cg_grads(const relres_params* p, const double* g_eps_cg, const double* g_sig_cg,
                                    double* g_eps_fg, double* g_sig_fg);

/*
 * Create a context on the current CUDA device for the lj/relres pair style of
 * Section 2.5: its parameters (FG eps and sigma per type, the hybrid flag, CG
 * eps and sigma per hybrid pair or Eq. 13 from group compositions) and the
 * four radii in the order r_s- <= r_s+ <= r_c- <= r_c+ the style requires.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).  The context
 * owns every internal device buffer and frees it in relres_destroy.
 * Errors: RELRES_ERR_ARG (invalid parameters, as relres_prepare_table),
 * RELRES_ERR_CUDA, RELRES_ERR_NOMEM.  *out is NULL on failure.
 */
relres_status relres_create(relres_ctx** out, const relres_params* p, void* cuda_stream);

/* Set atoms, masses, exclusions and bonded terms (replaces earlier ones).
 * A system has at least one atom.  Errors: RELRES_ERR_ARG (no atoms, index
 * out of range, asymmetric exclusions, type out of range), RELRES_ERR_NOMEM,
 * RELRES_ERR_CUDA. */
relres_status relres_set_topology(relres_ctx* ctx, const relres_topology* t);

/*
 * Bin atoms into cells and build both Verlet lists -- the two neighbour lists
 * of Section 2.6 that give RelRes its speed: the FG list over all atoms within
 * max r_s+ + skin, and the CG list over hybrid sites within max r_c+ +
 * skin_cg -- with exclusions removed.  d_pos: [n_atoms*3] device doubles, any
 * periodic image.  box: host double[3], orthorhombic edge lengths.
 * Sets the box used by later calls.  Synchronises the stream.
 * The CG skin is clamped to L/2 - r_c+ - 1e-6 when the box is small
 * (relres_get_stats reports it).  Grows list capacity as needed.
 * Errors: RELRES_ERR_STATE (no topology), RELRES_ERR_BOX (r_s+ + skin or r_c+
 * not below L/2), RELRES_ERR_LIST_OVERFLOW, RELRES_ERR_NONFINITE, RELRES_ERR_CUDA.
 */
relres_status relres_build_neighbors(relres_ctx* ctx, const double* d_pos, const double box[3]);

/*
 * One force evaluation at d_pos [n_atoms*3] (device): RelRes pair terms
 * (Eq. 20 over both lists) plus bonded terms.
 *   d_forces [n_atoms*3] device, overwritten (kcal/mol/A).
 *   d_energy [4] device or NULL: E_fg, E_cg, E_bonded, total, where E_fg + E_cg
 *            is the RelRes pair energy of Eq. 3 split exactly into the part
 *            on the FG list (r < r_s+) and the part on the CG list.
 *   d_virial [6] device or NULL: pair virial W_ab = sum_{i<j} (r_i-r_j)_a
 *            F_ij,b, order xx yy zz xy xz yz.
 * Lists are rebuilt first if any atom moved more than skin/2 since the last
 * build.  Synchronises the stream.
 * Errors: RELRES_ERR_STATE (no lists yet), RELRES_ERR_LIST_OVERFLOW,
 * RELRES_ERR_NONFINITE, RELRES_ERR_CUDA.
 */
relres_status relres_compute(relres_ctx* ctx, const double* d_pos, double* d_forces,
                             double* d_energy, double* d_virial);

/*
 * Molecular dynamics in the canonical ensemble, as the simulations of Section
 * 3.2 run it: n_steps of velocity Verlet (dt_fs) on d_pos/d_vel [n_atoms*3]
 * (device, updated in place; positions are returned wrapped into [0, L)).  Velocities
 * are A/fs.  Lists are rebuilt on the device whenever an atom has moved more
 * than skin/2.  t_target > 0 applies the CSVR thermostat (Bussi, Donadio &
 * Parrinello 2007) with time constant tau_fs after each step, N_f = 3N - 3,
 * drawing its random numbers from splitmix64 keyed by seed and the context's
 * step counter; t_target <= 0 is NVE.
 *   thermo_every > 0 and d_thermo != NULL: after every thermo_every-th step,
 *   row k of d_thermo [n_steps/thermo_every][RELRES_THERMO_COLS] receives
 *   E_fg E_cg E_bonded KE Wxx Wyy Wzz Wxy Wxz Wyz at that step.
 * A call given d_pos (and d_vel) still holding what the previous relres_step
 * returned continues from that call's end state (compared word for word on
 * the device): its forces are reused and, in FP32 mode with the same dt_fs,
 * its velocity state and last thermostat factors too, so that a run split
 * into calls of any length is the same bits as one call.  Arrays changed in
 * between are read: new positions get their forces computed, new velocities
 * replace the velocity state.
 * On RELRES_ERR_NONFINITE or RELRES_ERR_LIST_OVERFLOW the state is rolled
 * back to the last completed block of steps (blocks of up to 100 steps),
 * d_pos/d_vel receive it, and the error is returned.
 * Errors: RELRES_ERR_STATE, RELRES_ERR_LIST_OVERFLOW, RELRES_ERR_NONFINITE,
 * RELRES_ERR_ARG, RELRES_ERR_CUDA.
 */
relres_status relres_step(relres_ctx* ctx, int n_steps, double dt_fs, double* d_pos,
                          double* d_vel, double t_target, double tau_fs, uint64_t seed,
                          int thermo_every, double* d_thermo);

/* Set the step counter (thermostat random stream position), e.g. on resume. */
relres_status relres_set_step_counter(relres_ctx* ctx, long long step);

/* Statistics of the last build and counters (host struct). */
relres_status relres_get_stats(relres_ctx* ctx, relres_stats* out);

/*
 * Replace the LJ parameters of a context (eps_fg, sig_fg and the CG pair
 * parameters, explicit or by Eq. 13) without rebuilding its lists: the
 * differentiable form treats them as variables.  n_types, is_hybrid, mixing,
 * precision, shift, skin, every radius and the set of type pairs with
 * eps^CG > 0 must stay as at relres_create (RELRES_ERR_ARG otherwise, the
 * context unchanged).  Waits for the context stream.  Cached forces are
 * dropped (the next relres_step recomputes them).
 */
relres_status relres_set_params(relres_ctx* ctx, const relres_params* p);

/*
 * Backward pass of the RelRes pair interaction, Eq. 20 summed over pairs
 * (Eq. 3): the differentiable form of Section 2.5's potential.  For a scalar
 * L(E, F) of the pair energy E and the pair forces F (bonded terms are not
 * part of it), given
 *   grad_energy      dL/dE,
 *   d_grad_forces    [n_atoms*3] device, dL/dF_i (caller order), or NULL for 0,
 * at the positions d_pos ([n_atoms*3] device, as for relres_compute; the
 * lists are reused, or rebuilt if an atom moved more than half the skin), it
 * writes
 *   d_grad_pos       [n_atoms*3] device, dL/dx_i = grad_energy dE/dx_i -
 *                    sum_j h_ij (g_i - g_j) with the pair Hessian blocks
 *                    h_ij = u~'' rhat rhat^T + (u~'/r)(I - rhat rhat^T)
 *                    (a Hessian-vector product; u~'' exists in every region
 *                    thanks to the C2 smoothing of Eq. 7-8); may be NULL,
 *   grad_c           [n_types^2 * 4] host: per type pair (a*n_types + b)
 *                    dL/dC12 and dL/dC6 of the FG part, then of the CG part,
 *                    with C12 = 4 eps sig^12, C6 = 4 eps sig^6 (each part is
 *                    linear in them: Eq. 17-19 are linear in the potential);
 *                    record (a, b) collects half of every (a, b) pair and the
 *                    force terms of the type-a atoms; may be NULL,
 *   d_eps_fg, d_sig_fg  [n_types] host: dL/d eps_fg, dL/d sig_fg per type
 *                    through the mixing rule; may be NULL,
 *   d_eps_cg, d_sig_cg  [n_types^2] host: dL/d eps^CG, dL/d sig^CG per
 *                    record, the CG parameters taken as independent
 *                    variables (no chain through Eq. 13); may be NULL.
 * FP32 contexts evaluate in FP32 with FP64 totals, FP64 contexts in FP64.
 * Synchronises the context stream (the host outputs are read back).
 */
relres_status relres_backward(relres_ctx* ctx, const double* d_pos, const double* d_grad_forces,
                              double grad_energy, double* d_grad_pos, double* grad_c, double* d_eps_fg,
                              double* d_sig_fg, double* d_eps_cg, double* d_sig_cg);

/*
 * Step execution mode (an implementation choice; the paper has no
 * counterpart).  enable != 0 (the default) runs relres_step as one CUDA graph
 * per block of up to 100 steps: the list rebuild of every step is a
 * conditional node that a one-thread kernel opens only when the device-side
 * displacement trigger fired, so steps without a rebuild launch no binning or
 * list kernels.  The graph is captured on first use and reused while the
 * step arguments, the timing mode and the context's buffers stay the same
 * (re-captured otherwise).  enable == 0 launches the kernels on the stream
 * one by one, the rebuild kernels gated on the device flag.  Both modes give
 * bit-identical results.  Waits for the context stream; drops a captured
 * graph.
 */
relres_status relres_set_graphs(relres_ctx* ctx, int enable);

/*
 * Set the capacities of the FG and CG lists (entries per slot, rounded up to a
 * multiple of 8) and rebuild the lists at the current positions; a capacity
 * too small for them grows as on an overflow.  Later overflows inside
 * relres_step roll the step block back and grow the lists automatically, so
 * this only bounds the memory a caller is willing to start with.  Synchronous.
 */
relres_status relres_set_list_caps(relres_ctx* ctx, int cap_fg, int cap_cg);

/*
 * Testing and inspection (slow, synchronous): the entries of one neighbour
 * list as atom index pairs (i, j), i the list's owner, in list order.
 * which: 0 FG list, 1 CG list, 2 pruned FG list, 3 pruned CG list (as the
 * last build / pruning pass left them).  Writes min(*n_pairs, cap_pairs)
 * pairs to the host arrays h_i, h_j (may be NULL when cap_pairs == 0) and
 * the total count to *n_pairs.  Errors: RELRES_ERR_ARG, RELRES_ERR_STATE (no
 * lists yet; a pruned list with pruning off).
 */
relres_status relres_get_list(relres_ctx* ctx, int which, int* h_i, int* h_j, long long cap_pairs,
                              long long* n_pairs);

/*
 * Dynamic pruning of the two lists (Section 2.6 keeps the lists; pruning is a
 * property of this implementation).  The lists hold every pair within the
 * interaction cutoff (r_s+ for the FG list, r_c+ for the CG list) + skin at
 * the last build.  With delta > 0 a pruning pass copies, in list order, the
 * entries whose current distance is below the cutoff + delta into a second
 * pair of lists of the same capacity, and the pair kernels walk those.  A pass
 * follows every build and runs again at the first step after an atom has
 * moved more than delta/2 since the last pass.  The entries a pass drops
 * contribute exactly zero, so forces, virial and trajectories are the same
 * bits as without pruning when one thread walks each list (pair launch
 * configurations 0-2 of relres_set_pair_config) and the force sums are
 * running sums (RELRES_ACC_FP32, RELRES_ACC_FP64); the default compensated
 * sums add the entries four at a time, so there they agree to rounding, as do
 * the pair energies of the FP32 path (summed in an order that follows the
 * lists walked).  delta <= 0 turns pruning
 * off (the pair kernels then walk the full lists and the second pair of lists
 * is freed).  Default: delta = 0.5 A.  Rebuilds the lists at the current
 * positions if they exist.  Synchronous.  Errors: RELRES_ERR_ARG (null
 * context, non-finite delta).
 */
relres_status relres_set_prune(relres_ctx* ctx, double delta);

/*
 * Batches of independent replicas (an implementation choice; the paper has no
 * counterpart).  relres_batch_create groups n_ctx contexts (each created,
 * given its topology and neighbour lists as usual; any sizes and boxes; not
 * owned: destroy them after the batch).  relres_batch_step advances all of
 * them by n_steps like relres_step, with per-replica arrays
 *   d_pos[r], d_vel[r]   device positions / velocities of replica r,
 *   t_target[r], seed[r] thermostat target (<= 0: NVE) and random stream,
 *   d_thermo             NULL or per-replica thermo buffers (may be NULL),
 * and common dt_fs, tau_fs, thermo_every.  Each block of up to 100 steps is
 * one CUDA graph launch.  Where the replicas allow it (relres_batch_get_info)
 * each step is one drift, one pair and one force-sum launch covering every
 * replica (each kernel finds its replica from a table of block offsets), with
 * each replica's list rebuild a conditional node opened by one decide kernel;
 * otherwise every replica's block sits on its own branch of the graph.
 * Results are bit-identical to stepping each context alone with the same
 * arguments.  If any replica's list overflows, every replica returns to the
 * block start and the block is repeated with larger lists.  cuda_stream: the
 * stream the graphs run on (NULL: the batch creates its own).  Errors name the
 * replica (relres_batch_last_error).  Per-class kernel timing is not recorded
 * in batches.
 */
/*
 * Rates of the GPU this process runs on that the design of the library rests
 * on (not part of the method): FP32 and FP64 fused multiply-adds and
 * conversions from 64-bit integers to FP32 per clock per SM (issue-bound probe
 * kernels with independent chains), and the bandwidth of a plain float4 copy
 * from the first to the second half of d_scratch (count both the read and the
 * written bytes).  d_scratch: caller-owned device memory, 16-byte aligned, at
 * least 1 MiB and at least 2 KiB per SM; use a buffer well above the L2 size
 * (e.g. 2 GiB) for the copy to measure DRAM.  Runs on cuda_stream (NULL: the
 * default stream) and synchronises with it.  Errors: RELRES_ERR_ARG,
 * RELRES_ERR_CUDA.
 */
typedef struct relres_rates {
  double ffma_per_clk_sm, dfma_per_clk_sm, conv64_per_clk_sm;
  double copy_gbs;
  double fp32_tflops, fp64_tflops;  /* 2 flops per FMA at the SM count and the device's clock attribute */
  int sm_count, clock_mhz;
} relres_rates;
relres_status relres_measure_rates(void* d_scratch, size_t scratch_bytes, void* cuda_stream, relres_rates* out);

/*
 * Testing (synchronous): the reciprocals the pair kernels use in place of
 * correctly rounded division, on n inputs d_x[k] (device, FP64):
 *   d_out32[k]    = 1/x in FP32: hardware estimate of 1/float(x) plus one
 *                   Newton-Raphson step (results below the smallest normal
 *                   float are 0);
 *   d_out64[k]    = 1/x in FP64, and d_out64[n + k] = 1/sqrt(x): FP32
 *                   estimate plus one FP64 Newton-Raphson step.
 * d_out32 holds n floats, d_out64 2n doubles (device, caller-owned).
 * Errors: RELRES_ERR_ARG (null pointer, n < 0), RELRES_ERR_CUDA.
 */
relres_status relres_eval_recip(const double* d_x, float* d_out32, double* d_out64, int n, void* cuda_stream);

typedef struct relres_batch relres_batch;
relres_status relres_batch_create(relres_batch** out, relres_ctx* const* ctxs, int n_ctx, void* cuda_stream);
relres_status relres_batch_step(relres_batch* batch, int n_steps, double dt_fs, double* const* d_pos,
                                double* const* d_vel, const double* t_target, double tau_fs, const uint64_t* seed,
                                int thermo_every, double* const* d_thermo);
const char* relres_batch_last_error(relres_batch* batch);
/* *n_shared: how many replicas the last relres_batch_step ran in shared
 * launches (one drift, one pair and one force-sum launch per step covering all
 * of them, their list rebuilds in seven launches); the other replicas ran their
 * own kernels on branches of the same graph.  -1 before the first step. */
relres_status relres_batch_get_info(relres_batch* batch, int* n_shared);

/* Which replicas later relres_batch_step calls run in shared launches.
 * mode 1: every replica, which needs all of them with the same precision and
 * force accumulation and molecules of at most 256 atoms (RELRES_ERR_ARG at
 * the next step otherwise).  mode 0: none; every replica on its own branch of
 * the graph with its own kernels.  mode -1 (the default): the replicas of at
 * most RELRES_BATCH_SHARED_MAX_ATOMS atoms that share precision and force
 * accumulation (at least two); there the launch overhead of separate small
 * systems dominates, while a larger system runs faster with kernels of its
 * own (shared launches read each replica's arguments from device memory).
 * The pair kernel of shared launches runs one thread per atom in 256-thread
 * blocks whatever relres_set_pair_config chose.  Drops the captured graph.
 * Errors: RELRES_ERR_ARG (unknown mode). */
#define RELRES_BATCH_SHARED_MAX_ATOMS 16384
relres_status relres_batch_set_mode(relres_batch* batch, int mode);
void relres_batch_destroy(relres_batch* batch);

/*
 * Launch configuration of the forces-only FP32 pair kernel (an implementation
 * choice; the paper has no counterpart): config -1 (the default) lets the
 * first relres_step time every configuration -- threads sharing one atom's
 * list (1, 2, 4, 8) x block size -- on the context's own lists and keep the
 * fastest (systems under 20 000 atoms keep configuration 0; with list pruning
 * on only the one-thread configurations 0-2 are timed, since the others need a
 * separate pruning pass); config 0..6
 * fixes one (0: one thread per atom, 256 per block; 1, 2: one thread per
 * atom, 128, 512 per block; 3-6: 2, 4, 8, 2 threads per atom).  The choice is reported
 * in relres_stats.  Results agree within rounding (the summation order of an
 * atom's partners changes with the number of threads).
 */
relres_status relres_set_pair_config(relres_ctx* ctx, int config);

/*
 * Accumulation of each atom's pair-force sum in the FP32 pair kernels
 * (mode: relres_accumulation; an implementation choice, the paper names no
 * precision).  Applies to every later force evaluation and MD step of the
 * context; FP64 contexts ignore it.  Captured step graphs are dropped.
 * Errors: RELRES_ERR_ARG (null context, unknown mode).
 */
relres_status relres_set_force_accumulation(relres_ctx* ctx, int mode);

/*
 * Kernel timing.  enable != 0 makes relres_compute and relres_step record a
 * CUDA event pair on the context stream around every kernel class of
 * relres_timing_class and accumulate the elapsed times; enable == 0 stops it.
 * On the stream path the gated rebuild kernels are timed also when they find
 * nothing to do; in graph mode (relres_set_graphs) RELRES_T_REBUILD times the
 * decision kernel plus the conditional rebuild node (binning and both lists)
 * and RELRES_T_LISTS stays empty.  relres_set_timing always clears the totals.
 * relres_get_timings writes, for the first n classes, the total milliseconds
 * (ms[k]) and the number of timed launches (counts[k]; either may be NULL).
 */
relres_status relres_set_timing(relres_ctx* ctx, int enable);

/*
 * Sampled kernel timing: like relres_set_timing with enable != 0, but only the
 * classes whose bit (1 << relres_timing_class) is set in class_mask, and inside
 * relres_step only on steps k of a call with k % every == 0 (every >= 1).
 * Event records inside the step graphs cost a few microseconds each, so a
 * sparse sample times a kernel without slowing the steps around it.
 * class_mask 0 stops timing.  Clears the totals.
 */
relres_status relres_set_timing_sampled(relres_ctx* ctx, unsigned class_mask, int every);
relres_status relres_get_timings(relres_ctx* ctx, double* ms, long long* counts, int n);

/*
 * No-allocation pair evaluation (the paper has no counterpart: it is a
 * deployment aid).  For callers that cannot let a library allocate device
 * memory -- e.g. a host program that owns the GPU memory budget through its
 * own allocator and loads this library as a plug-in, or a loop in which the
 * device synchronisation of cudaMalloc/cudaFree is not allowed.  No context
 * is needed and nothing is allocated on the device: the scratch memory (the
 * type-pair table and per-block partial sums) is one file-scope static device
 * array, present on every GPU that loads the library until the process exits.
 *   p              parameters as for relres_create (only the pair terms are used).
 *   n_atoms        1..RELRES_STATIC_MAX_ATOMS, else RELRES_ERR_ARG.
 *   d_type         [n_atoms] device atom types.
 *   d_pos          [n_atoms*3] device positions (any periodic image).
 *   box            host double[3] orthorhombic edges; every interaction range
 *                  must be below half the box (else RELRES_ERR_BOX).
 *   d_excl_offsets, d_excl_index  device CSR exclusions as in relres_topology,
 *                  or both NULL.
 *   d_forces       [n_atoms*3] device output, overwritten: the RelRes pair
 *                  forces of Eq. 20 (no bonded terms), all pairs, FP64.
 *   d_energy       [1] device output or NULL: the pair energy (Eq. 3).
 *   d_virial       [6] device output or NULL: pair virial, as relres_compute.
 *   cuda_stream    cudaStream_t the work is enqueued on.
 * All calls on a GPU share the static array: calls whose work overlaps on the
 * GPU race on it and must be serialised by the caller.  Each call rewrites
 * every part of it that it reads and clears its bad-type flag first.  The
 * first call on each device (with that device current) looks up the array's
 * address.
 * Atom types are read on the device only: a type outside [0, n_types) is
 * never used to index the parameter table; that atom's forces and the
 * energy and virial of the call are written as NaN instead.  O(n_atoms^2)
 * work: meant for small systems.
 * Errors: RELRES_ERR_ARG, RELRES_ERR_BOX, RELRES_ERR_CUDA (returned for a
 * failure of this call's own copies or launches only).
 */
#define RELRES_STATIC_MAX_ATOMS 16384
relres_status relres_pair_forces_static(const relres_params* p, int n_atoms, const int* d_type,
                                        const double* d_pos, const double box[3],
                                        const int* d_excl_offsets, const int* d_excl_index,
                                        double* d_forces, double* d_energy, double* d_virial,
                                        void* cuda_stream);

/* Message for the last failure of ctx (owned by ctx; "" if none). */
const char* relres_last_error(relres_ctx* ctx);

/* Free everything the context owns.  NULL is a no-op. */
void relres_destroy(relres_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RELRES_H */
