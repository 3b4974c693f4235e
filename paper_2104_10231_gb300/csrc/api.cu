// C ABI of librelres (include/relres.h): context life cycle, topology, list
// builds, force evaluation and MD steps.  Host code only; kernels live in
// neighbor.cu, pair.cu and md.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <vector>

#include "relres_internal.h"

using namespace relres;

extern "C" {
static relres_status autotune_pairs(relres_ctx* c);  // defined with the C entry points below
static void drop_step_graph(relres_ctx* c);
}

namespace {

constexpr double kBoltz = 0.0019872042586408316;  // kcal/mol/K (R / 4184 J/kcal)

relres_status fail(relres_ctx* c, relres_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(c, RELRES_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}


unsigned long long morton3(unsigned x, unsigned y, unsigned z) {
  auto spread = [](unsigned v) {
    unsigned long long r = 0;
    for (int b = 0; b < 21; ++b) r |= (unsigned long long)((v >> b) & 1u) << (3 * b);
    return r;
  };
  return spread(x) | (spread(y) << 1) | (spread(z) << 2);
}

// Cells per axis: the largest count whose cells are at least r_list wide,
// cut into kXSplit slabs along x when every axis has four or more (see Grid).
relres_status setup_grid(relres_ctx* c, Grid* g, double rlist) {
  ++c->buf_gen;
  int nf[3];
  for (int d = 0; d < 3; ++d) nf[d] = std::max(1, int(std::floor(c->box[d] / rlist)));
  const int xs = (nf[0] >= 4 && nf[1] >= 4 && nf[2] >= 4) ? kXSplit : 1;
  const int n[3] = {nf[0] * xs, nf[1], nf[2]};
  if (g->d_rank_of && g->xsplit == xs && nf[0] == g->nf[0] && nf[1] == g->nf[1] && nf[2] == g->nf[2])
    return RELRES_OK;
  const long long ncf = (long long)nf[0] * nf[1] * nf[2];
  const long long nc = ncf * xs;
  if (nc > (1ll << 28)) return fail(c, RELRES_ERR_ARG, "too many cells");
  std::vector<std::pair<unsigned long long, int>> order;
  order.reserve(size_t(ncf));
  for (int x = 0; x < nf[0]; ++x)
    for (int y = 0; y < nf[1]; ++y)
      for (int z = 0; z < nf[2]; ++z) order.push_back({morton3(x, y, z), (x * nf[1] + y) * nf[2] + z});
  std::sort(order.begin(), order.end());
  std::vector<int> rank_full(static_cast<size_t>(ncf));
  for (size_t k = 0; k < order.size(); ++k) rank_full[size_t(order[k].second)] = int(k);
  std::vector<int> rank(static_cast<size_t>(nc));
  for (int x = 0; x < n[0]; ++x)
    for (int y = 0; y < n[1]; ++y)
      for (int z = 0; z < n[2]; ++z)
        rank[size_t((x * n[1] + y) * n[2] + z)] = rank_full[size_t(((x / xs) * nf[1] + y) * nf[2] + z)] * xs + x % xs;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = n[d];
    g->nf[d] = nf[d];
  }
  g->xsplit = xs;
  g->ncell = int(nc);
  g->ncell_full = int(ncf);
  g->ntile = int((nc + kScanTile - 1) / kScanTile);
  CK(dalloc(&g->d_rank_of, size_t(nc)));
  CK(dalloc(&g->d_start, size_t(nc) + 1));
  CK(dalloc(&g->d_count, size_t(nc)));
  CK(dalloc(&g->d_tile, size_t(g->ntile)));
  CK(cudaMemcpy(g->d_rank_of, rank.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
  CK(cudaMemset(g->d_count, 0, sizeof(int) * nc));
  CK(cudaMemset(g->d_start, 0, sizeof(int) * (nc + 1)));
  return RELRES_OK;
}

relres_status read_state(relres_ctx* c) {
  CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RELRES_OK;
}

// list capacity: a multiple of 8 (the lists are stored in chunks of 4), at
// most the number of possible partners rounded up
int round_cap(double x, int limit) {
  int v = int(std::ceil(x));
  v = (v + 7) / 8 * 8;
  const int lim = (std::max(8, limit) + 7) / 8 * 8;
  return std::max(8, std::min(v, lim));
}

relres_status alloc_lists(relres_ctx* c) {
  ++c->buf_gen;
  // list offsets are 32-bit inside the list kernel
  if (double(c->cap_fg) * c->n >= 2147483648.0 || double(c->cap_cg) * c->n_h >= 2147483648.0)
    return fail(c, RELRES_ERR_NOMEM, "neighbour list larger than 2^31 entries");
  CK(dalloc(&c->d_nbr_fg, size_t(c->cap_fg) * c->n));
  if (c->has_cg && c->n_h > 0) CK(dalloc(&c->d_nbr_cg, size_t(c->cap_cg) * c->n_h));
  // pruned lists: same layout and capacity (a pruned list is never longer)
  c->prune_on = c->prune_delta > 0.0;
  if (c->prune_on) {
    CK(dalloc(&c->d_nbr_fg_in, size_t(c->cap_fg) * c->n));
    CK(dalloc(&c->d_cnt_fg_in, size_t(c->n)));
    if (c->has_cg && c->n_h > 0) {
      CK(dalloc(&c->d_nbr_cg_in, size_t(c->cap_cg) * c->n_h));
      CK(dalloc(&c->d_cnt_cg_in, size_t(c->n_h)));
    }
  } else {
    dfree(c->d_nbr_fg_in);
    dfree(c->d_cnt_fg_in);
    dfree(c->d_nbr_cg_in);
    dfree(c->d_cnt_cg_in);
  }
  return RELRES_OK;
}

// Rebuild both lists at the current fixed-point positions, growing capacity
// until everything fits.
relres_status host_rebuild(relres_ctx* c) {
  CK(launch_flags_and(c, ~(unsigned)(F_REBUILD | F_PRUNE | F_OVERFLOW_FG | F_OVERFLOW_CG)));
  CK(launch_rebuild(c, nullptr));
  for (int attempt = 0; attempt < 4; ++attempt) {
    CK(launch_lists(c, nullptr));
    relres_status s = read_state(c);
    if (s != RELRES_OK) return s;
    const DevState& h = *c->h_state;
    if (h.flags & F_BADCELL) return fail(c, RELRES_ERR_CUDA, "cell binning produced an out-of-range index");
    const bool of = (h.flags & F_OVERFLOW_FG) != 0, oc = (h.flags & F_OVERFLOW_CG) != 0;
    if (!of && !oc) {
      c->last_max_fg = h.max_fg;
      c->last_max_cg = h.max_cg;
      c->last_mean_fg = c->n ? double(h.tot_fg) / c->n : 0.0;
      c->last_mean_cg = c->n_h ? double(h.tot_cg) / c->n_h : 0.0;
      c->have_lists = true;
      c->n_builds += 1;
      CK(launch_prune(c, nullptr));  // pruned lists at the same positions
      return RELRES_OK;
    }
    if (of) c->cap_fg = round_cap(h.max_fg * 1.2 + 8, c->n);
    if (oc) c->cap_cg = round_cap(h.max_cg * 1.2 + 8, c->n_h);
    s = alloc_lists(c);
    if (s != RELRES_OK) return s;
    CK(launch_flags_and(c, ~(unsigned)(F_OVERFLOW_FG | F_OVERFLOW_CG)));
    // list statistics are reset by the scan of a full rebuild; reset here too
    CK(cudaMemsetAsync(&c->d_state->max_fg, 0, 2 * sizeof(int), c->stream));
    CK(cudaMemsetAsync(&c->d_state->tot_fg, 0, 2 * sizeof(unsigned long long), c->stream));
  }
  return fail(c, RELRES_ERR_LIST_OVERFLOW, "neighbour list overflow after regrowth");
}

// ---- kernel timing: event pairs around each kernel class, read after a sync
cudaError_t tic(relres_ctx* c, int cls) {
  if (c->cap_marks) {  // capturing a step graph: the graph owns its (pre-created) events
    if (c->cap_used + 2 > c->cap_events->size()) return cudaErrorInvalidValue;
    relres_ctx::Mark m{cls, (*c->cap_events)[c->cap_used], (*c->cap_events)[c->cap_used + 1]};
    c->cap_used += 2;
    c->cap_marks->push_back(m);
    // external: a real event-record node (a plain record would only become a graph edge)
    return cudaEventRecordWithFlags(m.a, c->stream, cudaEventRecordExternal);
  }
  while (c->ev_used + 2 > c->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->ev_pool.push_back(e);
  }
  relres_ctx::Mark m{cls, c->ev_pool[c->ev_used], c->ev_pool[c->ev_used + 1]};
  c->ev_used += 2;
  c->marks.push_back(m);
  return cudaEventRecord(m.a, c->stream);
}

cudaError_t toc(relres_ctx* c) {
  if (c->cap_marks) return cudaEventRecordWithFlags(c->cap_marks->back().b, c->stream, cudaEventRecordExternal);
  return cudaEventRecord(c->marks.back().b, c->stream);
}

relres_status flush_timing(relres_ctx* c) {
  for (const relres_ctx::Mark& m : c->marks) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, m.a, m.b));
    c->t_ms[m.cls] += ms;
    c->t_cnt[m.cls] += 1;
  }
  c->marks.clear();
  c->ev_used = 0;
  return RELRES_OK;
}

static bool timed_now(const relres_ctx* c, int cls) {
  return c->timing && ((c->timing_mask >> cls) & 1u) && (c->cur_step % c->timing_every) == 0;
}

#define TIMED(cls, call)                     \
  do {                                       \
    const bool t_ = timed_now(c, cls);       \
    if (t_) CK(tic(c, cls));                 \
    CK(call);                                \
    if (t_) CK(toc(c));                      \
  } while (0)

// Lists valid at the positions already converted into d_xfx: a rebuild if an
// atom moved more than skin/2 since the last build, else a pruning pass if an
// atom moved more than delta/2 since the last one.
relres_status refresh_lists(relres_ctx* c) {
  if (c->h_state->flags & F_REBUILD) return host_rebuild(c);
  if (c->h_state->flags & F_PRUNE) {
    CK(launch_prune(c, nullptr));
    CK(launch_flags_and(c, ~(unsigned)F_PRUNE));
  }
  return RELRES_OK;
}

// Forces at the positions already converted into d_xfx (F_tot, FP64 copy optional).
relres_status forces_now(relres_ctx* c, int ev_mode, double* d_forces, double* d_energy,
                         double* d_virial) {
  relres_status s = read_state(c);
  if (s != RELRES_OK) return s;
  if (c->h_state->flags & F_NONFINITE) {
    CK(launch_flags_and(c, ~(unsigned)F_NONFINITE));
    return fail(c, RELRES_ERR_NONFINITE, "non-finite position");
  }
  s = refresh_lists(c);
  if (s != RELRES_OK) return s;
  if (!c->tuned) {
    s = autotune_pairs(c);
    if (s != RELRES_OK) return s;
  }
  CK(cudaMemsetAsync(c->d_acc, 0, sizeof(long long) * kNAcc, c->stream));
  TIMED(ev_mode == 1 ? RELRES_T_PAIR_EV : RELRES_T_PAIR, launch_pairs(c, ev_mode == 1));
  TIMED(RELRES_T_FINISH, launch_finish(c, ev_mode == 1, d_forces, nullptr));
  if (ev_mode == 1) TIMED(RELRES_T_THERMO, launch_reduce_out(c, d_energy, d_virial));
  s = read_state(c);
  if (s != RELRES_OK) return s;
  s = flush_timing(c);
  if (s != RELRES_OK) return s;
  if (c->h_state->flags & F_NONFINITE) {
    CK(launch_flags_and(c, ~(unsigned)F_NONFINITE));
    c->forces_valid = false;
    return fail(c, RELRES_ERR_NONFINITE, "non-finite force");
  }
  c->forces_valid = true;
  return RELRES_OK;
}

size_t force_bytes(const relres_ctx* c) { return size_t(c->n) * (c->fp64 ? 24 : 16); }



}  // namespace

extern "C" {

relres_status relres_create(relres_ctx** out, const relres_params* p, void* cuda_stream) {
  if (!out) return RELRES_ERR_ARG;
  *out = nullptr;
  relres_ctx* c = new (std::nothrow) relres_ctx();
  if (!c) return RELRES_ERR_NOMEM;
  const std::string e = build_pair_records(p, &c->recs);
  if (!e.empty()) {
    delete c;
    return RELRES_ERR_ARG;
  }
  c->prm = *p;
  c->n_types = p->n_types;
  c->eps_fg.assign(p->eps_fg, p->eps_fg + p->n_types);
  c->sig_fg.assign(p->sig_fg, p->sig_fg + p->n_types);
  c->is_hybrid.assign(p->is_hybrid, p->is_hybrid + p->n_types);
  // keep no caller pointers
  c->prm.eps_fg = c->eps_fg.data();
  c->prm.sig_fg = c->sig_fg.data();
  c->prm.is_hybrid = c->is_hybrid.data();
  c->prm.eps_cg = c->prm.sig_cg = nullptr;
  c->prm.group_comp = nullptr;
  c->prm.radii_pair = nullptr;
  c->fp64 = p->precision == RELRES_PREC_FP64;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  build_kernel_tables(c->recs, &c->tab_f, &c->tab_d);
  for (const PairRecord& r : c->recs) {
    c->rlist_fg_cut = std::max(c->rlist_fg_cut, r.rsp);
    if (r.eps_cg > 0.0) {
      c->has_cg = true;
      c->rlist_cg_cut = std::max(c->rlist_cg_cut, r.rcp);
    }
  }
  for (int t = 0; t < c->n_types; ++t)
    if (c->has_cg && c->is_hybrid[t]) c->hyb_mask |= 1 << t;
  const size_t tb = c->fp64 ? sizeof(PairTab<double>) * c->tab_d.size()
                            : sizeof(PairTab<float>) * c->tab_f.size();
  cudaError_t ce = cudaMalloc(&c->d_tab, tb);
  if (ce == cudaSuccess)
    ce = cudaMemcpy(c->d_tab, c->fp64 ? static_cast<const void*>(c->tab_d.data())
                                      : static_cast<const void*>(c->tab_f.data()),
                    tb, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_tabd, sizeof(PairTab<double>) * c->tab_d.size());
  if (ce == cudaSuccess)
    ce = cudaMemcpy(c->d_tabd, c->tab_d.data(), sizeof(PairTab<double>) * c->tab_d.size(),
                    cudaMemcpyHostToDevice);
  build_basis_tables(c->recs, p->shift, &c->basis_f, &c->basis_d);
  const size_t bb = c->fp64 ? sizeof(BasisTab<double>) * c->basis_d.size()
                            : sizeof(BasisTab<float>) * c->basis_f.size();
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_basis, bb);
  if (ce == cudaSuccess)
    ce = cudaMemcpy(c->d_basis, c->fp64 ? static_cast<const void*>(c->basis_d.data())
                                        : static_cast<const void*>(c->basis_f.data()),
                    bb, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_gc, sizeof(double) * 4 * c->recs.size());
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_state, sizeof(DevState));
  if (ce == cudaSuccess) ce = cudaMemset(c->d_state, 0, sizeof(DevState));
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_snap_state, sizeof(DevState));
  if (ce == cudaSuccess) ce = cudaMallocHost(&c->h_state, sizeof(DevState));
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_dummy, 256);
  if (ce == cudaSuccess) ce = cudaMemset(c->d_dummy, 0, 256);
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_acc, sizeof(long long) * kNAcc);
  if (ce == cudaSuccess) ce = cudaMemset(c->d_acc, 0, sizeof(long long) * kNAcc);
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_draws, sizeof(double) * 2 * kBlockSteps);
  if (ce == cudaSuccess) ce = cudaMemset(c->d_draws, 0, sizeof(double) * 2 * kBlockSteps);
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_open, sizeof(unsigned));
  if (ce == cudaSuccess) {
    const unsigned open = F_REBUILD;
    ce = cudaMemcpy(c->d_open, &open, sizeof(unsigned), cudaMemcpyHostToDevice);
  }
  if (ce != cudaSuccess) {
    relres_destroy(c);
    return ce == cudaErrorMemoryAllocation ? RELRES_ERR_NOMEM : RELRES_ERR_CUDA;
  }
  std::memset(c->h_state, 0, sizeof(DevState));
  *out = c;
  return RELRES_OK;
}

relres_status relres_set_topology(relres_ctx* c, const relres_topology* t) {
  if (!c) return RELRES_ERR_ARG;
  ++c->buf_gen;
  c->grad_n = 0;  // gradient buffers follow the atom counts
  if (!t || t->n_atoms < 1 || !t->type || !t->mass_by_type)
    return fail(c, RELRES_ERR_ARG, "topology needs n_atoms >= 1, type and mass_by_type");
  const int n = t->n_atoms;
  for (int k = 0; k < c->n_types; ++k)
    if (!(t->mass_by_type[k] > 0.0) || !std::isfinite(t->mass_by_type[k]))
      return fail(c, RELRES_ERR_ARG, "masses must be finite and > 0");
  for (int i = 0; i < n; ++i)
    if (t->type[i] < 0 || t->type[i] >= c->n_types) return fail(c, RELRES_ERR_ARG, "atom type out of range");
  // exclusions
  std::vector<int> eoff(size_t(n) + 1, 0), eidx;
  if ((t->excl_offsets == nullptr) != (t->excl_index == nullptr))
    return fail(c, RELRES_ERR_ARG, "excl_offsets and excl_index go together");
  if (t->excl_offsets) {
    if (t->excl_offsets[0] != 0) return fail(c, RELRES_ERR_ARG, "excl_offsets[0] must be 0");
    for (int i = 0; i < n; ++i) {
      if (t->excl_offsets[i + 1] < t->excl_offsets[i]) return fail(c, RELRES_ERR_ARG, "excl_offsets must be non-decreasing");
      eoff[i + 1] = t->excl_offsets[i + 1];
    }
    eidx.assign(t->excl_index, t->excl_index + eoff[n]);
    for (int i = 0; i < n; ++i)
      for (int k = eoff[i]; k < eoff[i + 1]; ++k) {
        const int j = eidx[k];
        if (j < 0 || j >= n || j == i) return fail(c, RELRES_ERR_ARG, "exclusion index out of range");
        bool sym = false;
        for (int m = eoff[j]; m < eoff[j + 1]; ++m) sym |= eidx[m] == i;
        if (!sym) return fail(c, RELRES_ERR_ARG, "exclusions must be symmetric");
      }
  }
  // bonded terms and the per-atom incident lists
  auto check_terms = [&](int count, const int* atoms, int width, const int* types, int ntypes) {
    if (count == 0) return true;
    if (!atoms || !types || ntypes < 1) return false;
    for (int k = 0; k < count; ++k) {
      if (types[k] < 0 || types[k] >= ntypes) return false;
      for (int w = 0; w < width; ++w)
        if (atoms[width * k + w] < 0 || atoms[width * k + w] >= n) return false;
    }
    return true;
  };
  if (t->n_bonds < 0 || t->n_angles < 0 || t->n_dihedrals < 0 ||
      !check_terms(t->n_bonds, t->bonds, 2, t->bond_type, t->n_bond_types) ||
      !check_terms(t->n_angles, t->angles, 3, t->angle_type, t->n_angle_types) ||
      !check_terms(t->n_dihedrals, t->dihedrals, 4, t->dihedral_type, t->n_dihedral_types))
    return fail(c, RELRES_ERR_ARG, "bonded term index or type out of range");
  if ((t->n_bonds && (!t->bond_k || !t->bond_r0)) || (t->n_angles && (!t->angle_k || !t->angle_theta0)) ||
      (t->n_dihedrals && !t->dihedral_k))
    return fail(c, RELRES_ERR_ARG, "bonded parameters missing");
  if (t->n_bonds + t->n_angles + t->n_dihedrals >= (1 << 28))
    return fail(c, RELRES_ERR_ARG, "too many bonded terms");
  // Terms of each kind in the order of their lowest atom (so that a run of
  // whole molecules owns a contiguous range of every kind, see segments below),
  // and the per-atom lists of incident terms in that order.
  auto order_by_min_atom = [&](int count, const int* atoms, int width) {
    std::vector<int> ord(size_t(std::max(0, count)));
    std::vector<int> lo(size_t(std::max(0, count)));
    for (int k = 0; k < count; ++k) {
      ord[k] = k;
      int m = atoms[width * k];
      for (int w = 1; w < width; ++w) m = std::min(m, atoms[width * k + w]);
      lo[k] = m;
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return lo[x] < lo[y]; });
    return ord;
  };
  const std::vector<int> ob = order_by_min_atom(t->n_bonds, t->bonds, 2);
  const std::vector<int> oa = order_by_min_atom(t->n_angles, t->angles, 3);
  const std::vector<int> od = order_by_min_atom(t->n_dihedrals, t->dihedrals, 4);
  std::vector<std::vector<int>> inc(static_cast<size_t>(n));
  std::vector<int4> hb(size_t(std::max(1, t->n_bonds))), ha(size_t(std::max(1, t->n_angles))),
      hd(size_t(std::max(1, t->n_dihedrals)));
  std::vector<int> hdt(size_t(std::max(1, t->n_dihedrals)), 0);
  // atoms spanned by each term (sorted order), for the segment boundaries
  std::vector<int> span_lo, span_hi;
  for (int k = 0; k < t->n_bonds; ++k) {
    const int q = ob[k];
    hb[k] = make_int4(t->bonds[2 * q], t->bonds[2 * q + 1], t->bond_type[q], 0);
    for (int r = 0; r < 2; ++r) inc[size_t(t->bonds[2 * q + r])].push_back((0 << 30) | (r << 28) | k);
    span_lo.push_back(std::min(hb[k].x, hb[k].y));
    span_hi.push_back(std::max(hb[k].x, hb[k].y));
  }
  for (int k = 0; k < t->n_angles; ++k) {
    const int q = oa[k];
    ha[k] = make_int4(t->angles[3 * q], t->angles[3 * q + 1], t->angles[3 * q + 2], t->angle_type[q]);
    for (int r = 0; r < 3; ++r) inc[size_t(t->angles[3 * q + r])].push_back((1 << 30) | (r << 28) | k);
    span_lo.push_back(std::min({ha[k].x, ha[k].y, ha[k].z}));
    span_hi.push_back(std::max({ha[k].x, ha[k].y, ha[k].z}));
  }
  for (int k = 0; k < t->n_dihedrals; ++k) {
    const int q = od[k];
    hd[k] = make_int4(t->dihedrals[4 * q], t->dihedrals[4 * q + 1], t->dihedrals[4 * q + 2],
                      t->dihedrals[4 * q + 3]);
    hdt[k] = t->dihedral_type[q];
    for (int r = 0; r < 4; ++r) inc[size_t(t->dihedrals[4 * q + r])].push_back((2 << 30) | (r << 28) | k);
    span_lo.push_back(std::min({hd[k].x, hd[k].y, hd[k].z, hd[k].w}));
    span_hi.push_back(std::max({hd[k].x, hd[k].y, hd[k].z, hd[k].w}));
  }
  std::vector<int> ioff(size_t(n) + 1, 0), iall;
  for (int i = 0; i < n; ++i) {
    ioff[i + 1] = ioff[i] + int(inc[i].size());
    iall.insert(iall.end(), inc[i].begin(), inc[i].end());
  }
  // Segments: runs of at most kSegAtoms atoms that no bonded term crosses,
  // each with the contiguous range of its terms of every kind.  The fused
  // bonded + force-sum kernel gives one block to each segment; without a valid
  // segmentation (a molecule larger than a segment) the two-kernel path runs.
  std::vector<int> seg;
  int seg_slots = 0;
  bool seg_ok = true;
  {
    std::vector<int> cross(size_t(n) + 2, 0);  // > 0: a term spans the boundary before atom a
    for (size_t k = 0; k < span_lo.size(); ++k) {
      cross[size_t(span_lo[k]) + 1] += 1;
      cross[size_t(span_hi[k]) + 1] -= 1;
    }
    for (int a = 1; a <= n; ++a) cross[a] += cross[a - 1];
    auto first_ge = [](const std::vector<int4>& v, int count, int which, int atom) {
      int lo = 0, hi = count;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        const int4 q = v[mid];
        int m = std::min(q.x, q.y);
        if (which >= 1) m = std::min(m, q.z);
        if (which >= 2) m = std::min(m, q.w);
        if (m < atom) lo = mid + 1; else hi = mid;
      }
      return lo;
    };
    int a0 = 0;
    while (a0 < n && seg_ok) {
      int a1 = std::min(n, a0 + kSegAtoms);
      while (a1 > a0 && a1 < n && cross[a1] > 0) --a1;
      if (a1 == a0) {
        seg_ok = false;
        break;
      }
      const int b0 = first_ge(hb, t->n_bonds, 0, a0), b1 = first_ge(hb, t->n_bonds, 0, a1);
      const int g0 = first_ge(ha, t->n_angles, 1, a0), g1 = first_ge(ha, t->n_angles, 1, a1);
      const int d0 = first_ge(hd, t->n_dihedrals, 2, a0), d1 = first_ge(hd, t->n_dihedrals, 2, a1);
      seg.insert(seg.end(), {a0, a1, b0, b1, g0, g1, d0, d1, a0});
      seg_slots = std::max(seg_slots, 2 * (b1 - b0) + 3 * (g1 - g0) + 4 * (d1 - d0));
      a0 = a1;
    }
    // Prototypes: a segment whose term records and incident-term lists, taken
    // relative to its first atom and first term of each kind, equal those of
    // an earlier segment reads that segment's records instead of its own (the
    // same terms in the same order, so the same arithmetic): in a liquid of
    // identical molecules every full segment shares one prototype, whose
    // records stay in L1/L2.
    if (seg_ok) {
      std::map<std::vector<int>, int> first;  // normalised segment -> its first segment
      std::vector<int> key;
      for (size_t q = 0; q * kSegRec < seg.size(); ++q) {
        int* r = &seg[q * kSegRec];
        const int s0 = r[0], s1 = r[1], rb0 = r[2], rb1 = r[3], rg0 = r[4], rg1 = r[5], rd0 = r[6], rd1 = r[7];
        key.assign({s1 - s0, rb1 - rb0, rg1 - rg0, rd1 - rd0});
        for (int k = rb0; k < rb1; ++k) key.insert(key.end(), {hb[k].x - s0, hb[k].y - s0, hb[k].z});
        for (int k = rg0; k < rg1; ++k) key.insert(key.end(), {ha[k].x - s0, ha[k].y - s0, ha[k].z - s0, ha[k].w});
        for (int k = rd0; k < rd1; ++k)
          key.insert(key.end(), {hd[k].x - s0, hd[k].y - s0, hd[k].z - s0, hd[k].w - s0, hdt[k]});
        for (int i = s0; i < s1; ++i) {
          key.push_back(ioff[i + 1] - ioff[i]);
          for (int m = ioff[i]; m < ioff[i + 1]; ++m) {
            const int item = iall[m], kind = (item >> 30) & 3, term = item & 0x0fffffff;
            const int rel = term - (kind == 0 ? rb0 : (kind == 1 ? rg0 : rd0));
            key.push_back((item & ~0x0fffffff) ^ rel);
          }
        }
        const auto it = first.find(key);
        if (it == first.end()) {
          first.emplace(key, int(q));
          continue;
        }
        const int* p0 = &seg[size_t(it->second) * kSegRec];
        for (int w = 2; w < 8; ++w) r[w] = p0[w];
        r[8] = p0[0];
      }
      c->n_seg_proto = int(first.size());
    }
    // shared memory of the segment kernels: term slots (float4 or 3 doubles)
    // plus the segment's positions in the drift kernel
    const size_t slot_bytes = c->fp64 ? 24 : 16;
    if (size_t(std::max(1, seg_slots)) * slot_bytes + 24 * size_t(kSegAtoms) > kSegSmemMax) seg_ok = false;
  }
  std::vector<double> bp(2 * size_t(std::max(1, t->n_bond_types)), 0.0),
      ap(2 * size_t(std::max(1, t->n_angle_types)), 0.0), dp(4 * size_t(std::max(1, t->n_dihedral_types)), 0.0);
  for (int k = 0; k < t->n_bond_types && t->n_bonds; ++k) {
    bp[2 * k] = t->bond_k[k];
    bp[2 * k + 1] = t->bond_r0[k];
  }
  for (int k = 0; k < t->n_angle_types && t->n_angles; ++k) {
    ap[2 * k] = t->angle_k[k];
    ap[2 * k + 1] = t->angle_theta0[k];
  }
  for (int k = 0; k < 4 * t->n_dihedral_types && t->n_dihedrals; ++k) dp[k] = t->dihedral_k[k];

  c->n = n;
  c->excl_window = 0;
  for (int i = 0; i < n; ++i)
    for (int m = eoff[i]; m < eoff[i + 1]; ++m) c->excl_window = std::max(c->excl_window, std::abs(eidx[m] - i));
  c->h_type.assign(t->type, t->type + n);
  c->mass_by_type.assign(t->mass_by_type, t->mass_by_type + c->n_types);
  c->n_h = 0;
  std::vector<int> rank_cg(static_cast<size_t>(n), -1);
  for (int i = 0; i < n; ++i)
    if ((c->hyb_mask >> c->h_type[i]) & 1) ++c->n_h;
  c->n_bonds = t->n_bonds;
  c->n_angles = t->n_angles;
  c->n_dih = t->n_dihedrals;
  const int nh = std::max(1, c->n_h);
  const size_t fb = size_t(n) * (c->fp64 ? 24 : 16);
  CK(dalloc(&c->d_type, n));
  CK(dalloc(&c->d_cdt, RELRES_MAX_TYPES));
  CK(dalloc(&c->d_cdt_ff, RELRES_MAX_TYPES));
  CK(dalloc(&c->d_kec, RELRES_MAX_TYPES));
  CK(dalloc(&c->d_mass, RELRES_MAX_TYPES));
  CK(dalloc(&c->d_excl_off, size_t(n) + 1));
  CK(dalloc(&c->d_excl_idx, std::max<size_t>(1, eidx.size())));
  dfree(c->d_excl_mask);
  if (c->excl_window <= kExclMaskHalf) {
    std::vector<unsigned> em(size_t(n), 1u << kExclMaskHalf);  // the atom itself
    for (int i = 0; i < n; ++i)
      for (int m = eoff[i]; m < eoff[i + 1]; ++m) em[i] |= 1u << (eidx[m] - i + kExclMaskHalf);
    CK(dalloc(&c->d_excl_mask, size_t(n)));
    CK(cudaMemcpy(c->d_excl_mask, em.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice));
  }
  CK(dalloc(&c->d_bonds, hb.size()));
  CK(dalloc(&c->d_angles, ha.size()));
  CK(dalloc(&c->d_dihs, hd.size()));
  CK(dalloc(&c->d_dih_type, hdt.size()));
  CK(dalloc(&c->d_bond_par, bp.size()));
  CK(dalloc(&c->d_angle_par, ap.size()));
  CK(dalloc(&c->d_dih_par, dp.size()));
  std::vector<float> bfp(4 * (bp.size() / 2), 0.f), afp(8 * (ap.size() / 2), 0.f);
  for (size_t k = 0; k < bp.size() / 2; ++k) {
    bfp[4 * k] = float(bp[2 * k]);
    bfp[4 * k + 1] = float(bp[2 * k + 1]);
    bfp[4 * k + 2] = float(bp[2 * k + 1] - double(bfp[4 * k + 1]));
  }
  for (size_t k = 0; k < ap.size() / 2; ++k) {
    const double t0 = ap[2 * k + 1], c0 = std::cos(t0), s0 = std::sin(t0);
    afp[8 * k] = float(ap[2 * k]);
    afp[8 * k + 1] = float(t0);
    afp[8 * k + 2] = float(c0);
    afp[8 * k + 3] = float(c0 - double(afp[8 * k + 2]));
    afp[8 * k + 4] = float(s0);
    afp[8 * k + 5] = float(s0 - double(afp[8 * k + 4]));
  }
  CK(dalloc(&c->d_bond_fpar, bfp.size()));
  CK(dalloc(&c->d_angle_fpar, afp.size()));
  CK(cudaMemcpy(c->d_bond_fpar, bfp.data(), sizeof(float) * bfp.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_angle_fpar, afp.data(), sizeof(float) * afp.size(), cudaMemcpyHostToDevice));
  CK(dalloc(&c->d_inc_off, ioff.size()));
  CK(dalloc(&c->d_inc, std::max<size_t>(1, iall.size())));
  CK(dalloc(&c->d_xfx, 3 * size_t(n)));
  CK(dalloc(&c->d_ref, size_t(n)));
  CK(dalloc(&c->d_ref_p, size_t(n)));
  CK(dalloc(&c->d_cell_fg, size_t(n)));
  CK(dalloc(&c->d_cell_cg, size_t(n)));
  CK(dalloc(&c->d_slot_fg, size_t(n)));
  CK(dalloc(&c->d_slot_cg, size_t(n)));
  CK(dalloc(&c->d_perm_fg, size_t(n)));
  CK(dalloc(&c->d_rank_fg, size_t(n)));
  CK(dalloc(&c->d_perm_cg, size_t(nh)));
  CK(dalloc(&c->d_rank_cg, size_t(n)));
  CK(dalloc(&c->d_pos_fg, size_t(n)));
  CK(dalloc(&c->d_pos_cg, size_t(nh)));
  if (c->fp64) {
    CK(dalloc(&c->d_pos_fg64, size_t(n)));
    CK(dalloc(&c->d_pos_cg64, size_t(nh)));
  }
  CK(dalloc(&c->d_cnt_fg, size_t(n)));
  CK(dalloc(&c->d_cnt_cg, size_t(nh)));
  CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_f_fg), fb));
  CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_f_cg), fb));
  CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_f_tot), fb));
  CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_f_bond), fb));
  CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_snap_f), fb));
  CK(dalloc(&c->d_snap_x, 3 * size_t(n)));
  CK(dalloc(&c->d_snap_v, 3 * size_t(n)));
  CK(dalloc(&c->d_uff, 3 * size_t(n)));
  CK(dalloc(&c->d_pos_ret, 3 * size_t(n)));
  CK(dalloc(&c->d_vel_ret, 3 * size_t(n)));
  c->io_valid = false;
  const size_t n_slots = 2 * size_t(c->n_bonds) + 3 * size_t(c->n_angles) + 4 * size_t(c->n_dih);
  CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_tf),
            std::max<size_t>(1, n_slots) * (c->fp64 ? 24 : 16)));
  CK(cudaMemcpy(c->d_type, c->h_type.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_mass, c->mass_by_type.data(), sizeof(double) * c->n_types, cudaMemcpyHostToDevice));
  CK(cudaMemset(c->d_cdt, 0, sizeof(double) * RELRES_MAX_TYPES));
  CK(cudaMemcpy(c->d_excl_off, eoff.data(), sizeof(int) * eoff.size(), cudaMemcpyHostToDevice));
  if (!eidx.empty()) CK(cudaMemcpy(c->d_excl_idx, eidx.data(), sizeof(int) * eidx.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_bonds, hb.data(), sizeof(int4) * hb.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_angles, ha.data(), sizeof(int4) * ha.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_dihs, hd.data(), sizeof(int4) * hd.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_dih_type, hdt.data(), sizeof(int) * hdt.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_bond_par, bp.data(), sizeof(double) * bp.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_angle_par, ap.data(), sizeof(double) * ap.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_dih_par, dp.data(), sizeof(double) * dp.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_inc_off, ioff.data(), sizeof(int) * ioff.size(), cudaMemcpyHostToDevice));
  if (!iall.empty()) CK(cudaMemcpy(c->d_inc, iall.data(), sizeof(int) * iall.size(), cudaMemcpyHostToDevice));
  c->seg_ok = seg_ok && !seg.empty();
  c->n_seg = int(seg.size() / kSegRec);
  c->seg_slots = std::max(1, seg_slots);
  if (c->seg_ok) {
    CK(dalloc(&c->d_seg, seg.size()));
    CK(cudaMemcpy(c->d_seg, seg.data(), sizeof(int) * seg.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(c->d_rank_cg, rank_cg.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CK(cudaMemset(c->d_f_cg, 0, fb));
  c->have_topo = true;
  c->have_lists = false;
  c->consts_dt = 0.0;  // masses may have changed
  c->forces_valid = false;
  c->cap_fg = c->cap_cg = 0;
  return RELRES_OK;
}

relres_status relres_build_neighbors(relres_ctx* c, const double* d_pos, const double box[3]) {
  if (c) ++c->buf_gen;
  if (!c) return RELRES_ERR_ARG;
  if (!c->have_topo) return fail(c, RELRES_ERR_STATE, "relres_set_topology first");
  if (!d_pos || !box) return fail(c, RELRES_ERR_ARG, "d_pos and box are required");
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) return fail(c, RELRES_ERR_ARG, "box edges must be finite and > 0");
  const double lmin = std::min(box[0], std::min(box[1], box[2]));
  const double rfg = c->rlist_fg_cut + c->prm.skin;
  if (!(rfg < 0.5 * lmin)) return fail(c, RELRES_ERR_BOX, "r_s+ + skin must be below half the box");
  double skin_cg = c->prm.skin;
  if (c->has_cg) {
    if (!(c->rlist_cg_cut < 0.5 * lmin)) return fail(c, RELRES_ERR_BOX, "r_c+ must be below half the box");
    skin_cg = std::min(skin_cg, 0.5 * lmin - c->rlist_cg_cut - 1e-6);
  }
  const bool same_box = c->have_box && box[0] == c->box[0] && box[1] == c->box[1] && box[2] == c->box[2];
  for (int d = 0; d < 3; ++d) c->box[d] = box[d];
  c->skin_cg = skin_cg;
  c->have_box = true;
  if (!same_box) c->forces_valid = false;
  relres_status s = setup_grid(c, &c->gfg, rfg);
  if (s != RELRES_OK) return s;
  if (c->has_cg && c->n_h > 0) {
    s = setup_grid(c, &c->gcg, c->rlist_cg_cut + skin_cg);
    if (s != RELRES_OK) return s;
  }
  if (c->cap_fg == 0) {
    const double vol = box[0] * box[1] * box[2];
    const double pi43 = 4.18879020478639;
    c->cap_fg = round_cap(1.3 * pi43 * rfg * rfg * rfg * c->n / vol + 24, c->n);
    const double rcg = c->rlist_cg_cut + skin_cg;
    c->cap_cg = round_cap(1.3 * pi43 * rcg * rcg * rcg * c->n_h / vol + 24, c->n_h);
    s = alloc_lists(c);
    if (s != RELRES_OK) return s;
  }
  const bool had = c->have_lists;
  c->have_lists = false;  // no sorted scatter before the first pack
  c->io_valid = false;
  CK(launch_convert(c, d_pos));
  c->have_lists = had;
  s = read_state(c);
  if (s != RELRES_OK) return s;
  if (c->h_state->flags & F_NONFINITE) {
    CK(launch_flags_and(c, ~(unsigned)F_NONFINITE));
    return fail(c, RELRES_ERR_NONFINITE, "non-finite position");
  }
  c->forces_valid = false;
  return host_rebuild(c);
}

relres_status relres_compute(relres_ctx* c, const double* d_pos, double* d_forces, double* d_energy,
                             double* d_virial) {
  if (!c) return RELRES_ERR_ARG;
  if (!c->have_lists) return fail(c, RELRES_ERR_STATE, "relres_build_neighbors first");
  if (!d_pos || !d_forces) return fail(c, RELRES_ERR_ARG, "d_pos and d_forces are required");
  c->io_valid = false;
  CK(launch_convert(c, d_pos));
  return forces_now(c, (d_energy || d_virial) ? 1 : 0, d_forces, d_energy, d_virial);
}

// ---- autotuner of the forces-only pair kernel: every launch configuration
// (threads per slot x block size) is timed on the context's own lists and the
// fastest is kept.  Runs once per context, at the first relres_step (the step
// graph bakes the choice in); forces-only launches write only the per-list
// force scratch, which the next evaluation overwrites.
static relres_status autotune_pairs(relres_ctx* c) {
  c->tuned = true;
  if (c->tune_mode >= 0 || c->fp64 || c->n < 20000) {
    c->pair_cfg = c->tune_mode >= 0 ? c->tune_mode : 0;
    return RELRES_OK;
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_cfg = 0;
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < kNPairConfigs && err == cudaSuccess; ++k) {
    // with pruning, launches with one thread per slot prune as they go; the
    // others need a separate pruning pass, so they are not candidates
    if (c->prune_on && kPairConfigs[k].tpa != 1) continue;
    c->pair_cfg = k;
    err = launch_pairs(c, false);  // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) err = launch_pairs(c, false);
    if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < best) {
      best = ms;
      best_cfg = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->pair_cfg = best_cfg;
  CK(err);
  return RELRES_OK;
}

relres_status relres_set_list_caps(relres_ctx* c, int cap_fg, int cap_cg) {
  if (!c || cap_fg < 1 || cap_cg < 1) return RELRES_ERR_ARG;
  if (!c->have_lists) return fail(c, RELRES_ERR_STATE, "relres_build_neighbors first");
  CK(cudaStreamSynchronize(c->stream));
  c->cap_fg = round_cap(cap_fg, c->n);
  c->cap_cg = round_cap(cap_cg, c->n_h);
  relres_status s = alloc_lists(c);
  if (s != RELRES_OK) return s;
  s = host_rebuild(c);  // at the current positions; grows a capacity that is too small
  if (s != RELRES_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  return RELRES_OK;
}

relres_status relres_get_list(relres_ctx* c, int which, int* h_i, int* h_j, long long cap_pairs,
                              long long* n_pairs) {
  if (!c || !n_pairs || which < 0 || which > 3 || cap_pairs < 0 || (cap_pairs > 0 && (!h_i || !h_j)))
    return RELRES_ERR_ARG;
  if (!c->have_lists) return fail(c, RELRES_ERR_STATE, "relres_build_neighbors first");
  const bool cg = (which & 1) != 0, pruned = which >= 2;
  if (pruned && !c->prune_on) return fail(c, RELRES_ERR_STATE, "pruning is off");
  const int nslots = cg ? ((c->has_cg && c->n_h > 0) ? c->n_h : 0) : c->n;
  *n_pairs = 0;
  if (nslots == 0) return RELRES_OK;
  const int cap = cg ? c->cap_cg : c->cap_fg;
  const int* d_nbr = pruned ? (cg ? c->d_nbr_cg_in : c->d_nbr_fg_in) : (cg ? c->d_nbr_cg : c->d_nbr_fg);
  const int* d_cnt = pruned ? (cg ? c->d_cnt_cg_in : c->d_cnt_fg_in) : (cg ? c->d_cnt_cg : c->d_cnt_fg);
  const int* d_perm = cg ? c->d_perm_cg : c->d_perm_fg;
  const size_t ns = static_cast<size_t>(nslots);
  std::vector<int> cnt(ns), perm(ns), nbr(static_cast<size_t>(cap) * ns);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(cnt.data(), d_cnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(perm.data(), d_perm, sizeof(int) * perm.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(nbr.data(), d_nbr, sizeof(int) * nbr.size(), cudaMemcpyDeviceToHost));
  long long k = 0;
  for (int sl = 0; sl < nslots; ++sl)
    for (int e = 0; e < std::min(cnt[sl], cap); ++e, ++k) {
      if (k < cap_pairs) {
        const int j = nbr[(size_t(e >> 2) * nslots + sl) * 4 + (e & 3)];
        h_i[k] = perm[sl];
        h_j[k] = (j >= 0 && j < nslots) ? perm[j] : -1;
      }
    }
  *n_pairs = k;
  return RELRES_OK;
}

relres_status relres_set_prune(relres_ctx* c, double delta) {
  if (!c || !std::isfinite(delta)) return RELRES_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->prune_delta = delta > 0.0 ? delta : 0.0;
  if (!c->have_lists) {  // applied at the first build
    c->prune_on = c->prune_delta > 0.0;
    return RELRES_OK;
  }
  relres_status s = alloc_lists(c);
  if (s != RELRES_OK) return s;
  s = host_rebuild(c);  // both lists at the current positions
  if (s != RELRES_OK) return s;
  c->forces_valid = false;
  CK(cudaStreamSynchronize(c->stream));
  return RELRES_OK;
}

relres_status relres_set_force_accumulation(relres_ctx* c, int mode) {
  if (!c) return RELRES_ERR_ARG;
  if (mode != RELRES_ACC_FP32 && mode != RELRES_ACC_COMPENSATED && mode != RELRES_ACC_FP64)
    return fail(c, RELRES_ERR_ARG, "unknown force accumulation mode");
  CK(cudaStreamSynchronize(c->stream));
  c->force_acc = mode;
  drop_step_graph(c);
  ++c->buf_gen;  // batch graphs bake the launches in too
  return RELRES_OK;
}

relres_status relres_set_pair_config(relres_ctx* c, int config) {
  if (!c || config < -1 || config >= kNPairConfigs) return RELRES_ERR_ARG;
  c->tune_mode = config;
  c->tuned = false;
  c->pair_cfg = config >= 0 ? config : 0;
  return RELRES_OK;
}

// ---- relres_step: one block of steps, recorded either on the stream (the
// rebuild kernels gated on the device flag) or into a CUDA graph (the
// rebuild of each step behind a conditional node).

static void drop_one_graph(relres_ctx::StepGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (cudaEvent_t e : g.events) cudaEventDestroy(e);
  g = relres_ctx::StepGraph{};
}

static void drop_step_graph(relres_ctx* c) {
  for (relres_ctx::StepGraph& g : c->sgs) drop_one_graph(g);
  c->sgs.clear();
  c->sg_cur = -1;
}

// A conditional (IF) node added to the graph being captured on c->stream
// after its current dependencies; `body` records the node's body on a second
// stream (ungated launches).
static relres_status add_conditional(relres_ctx* c, cudaGraphConditionalHandle h,
                                     const std::function<cudaError_t()>& body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c->stream, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return fail(c, RELRES_ERR_CUDA, "stream is not capturing");
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &cp));
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  const cudaStream_t main = c->stream;
  CK(cudaStreamBeginCaptureToGraph(c->body_stream, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  c->stream = c->body_stream;
  const cudaError_t e1 = body();
  c->stream = main;
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->body_stream, &out);
  CK(e1);
  CK(e2);
  CK(cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return RELRES_OK;
}

// The conditional rebuild node of one step (binning + lists).  One one-thread
// kernel sets its flag and, with a separate pruning pass (pruning on, several
// threads per slot), the flag of the pruning node (*hp: a rebuild or the
// pruning trigger fired), which record_pairs adds after it.
static relres_status add_rebuild_node(relres_ctx* c, cudaGraphConditionalHandle* hp) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(c->stream, &st, nullptr, &g, nullptr, nullptr, nullptr));
  if (st != cudaStreamCaptureStatusActive) return fail(c, RELRES_ERR_CUDA, "stream is not capturing");
  cudaGraphConditionalHandle h;
  *hp = 0;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  const bool separate = c->prune_on && !pairs_prune(c);
  if (separate) CK(cudaGraphConditionalHandleCreate(hp, g, 0, cudaGraphCondAssignDefault));
  CK(launch_decide(c, h, *hp, separate ? 1 : 0));
  return add_conditional(c, h, [c]() {
    const cudaError_t e = launch_rebuild(c, c->d_open);
    return e == cudaSuccess ? launch_lists(c, c->d_open) : e;
  });
}

// The pair evaluation of one step.  With pruning and one thread per slot the
// pair kernel itself prunes on the steps that need it (it reads the device
// flags); with several threads per slot a separate pruning pass runs first on
// those steps (graph: a conditional node; stream: a launch gated on the flags).
static relres_status record_pairs(relres_ctx* c, bool ev, bool graph, cudaGraphConditionalHandle hp) {
  if (c->prune_on && !pairs_prune(c)) {
    if (graph) {
      const bool t_ = timed_now(c, RELRES_T_PRUNE);
      if (t_) CK(tic(c, RELRES_T_PRUNE));
      relres_status s = add_conditional(c, hp, [c]() { return launch_prune(c, c->d_open); });
      if (s != RELRES_OK) return s;
      if (t_) CK(toc(c));
    } else {
      TIMED(RELRES_T_PRUNE, launch_prune(c, &c->d_state->flags));
    }
  }
  TIMED(ev ? RELRES_T_PAIR_EV : RELRES_T_PAIR, launch_pairs(c, ev));
  return RELRES_OK;
}

// The work of one block of blk steps starting after `done` steps of the call.
static relres_status record_block(relres_ctx* c, const StepParams& sp, double* d_vel, int blk, int done,
                                  bool graph) {
  const unsigned* gate = &c->d_state->flags;
  const size_t xb = sizeof(unsigned long long) * 3 * size_t(c->n), vb = sizeof(double) * 3 * size_t(c->n);
  CK(cudaMemcpyAsync(c->d_snap_x, c->d_xfx, xb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_snap_v, vel_state(c, d_vel), vb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_snap_f, c->d_f_tot, force_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_snap_state, c->d_state, sizeof(DevState), cudaMemcpyDeviceToDevice, c->stream));
  CK(launch_csvr_draws(c, sp, blk));
  for (int k = 0; k < blk; ++k) {
    c->cur_step = done + k;
    // energy steps are known here: the device sets DevState::ev by the same rule
    const bool ev_step = sp.thermo_every > 0 && ((done + k + 1) % sp.thermo_every) == 0;
    TIMED(RELRES_T_DRIFT, launch_drift(c, sp, d_vel, ev_step, k > 0));
    cudaGraphConditionalHandle hp = 0;
    if (graph) {
      const bool t_ = timed_now(c, RELRES_T_REBUILD);
      if (t_) CK(tic(c, RELRES_T_REBUILD));
      relres_status s = add_rebuild_node(c, &hp);
      if (s != RELRES_OK) return s;
      if (t_) CK(toc(c));
    } else {
      TIMED(RELRES_T_REBUILD, launch_rebuild(c, gate));
      TIMED(RELRES_T_LISTS, launch_lists(c, gate));
    }
    relres_status sp_ = record_pairs(c, ev_step, graph, hp);
    if (sp_ != RELRES_OK) return sp_;
    if (step_segments(c)) {  // bonded forces came with the drift; thermostat in k_sum's last block
      TIMED(RELRES_T_FINISH, launch_end_of_step(c, sp, k, ev_step, d_vel));
    } else {
      TIMED(RELRES_T_FINISH, launch_finish(c, ev_step, nullptr, d_vel));
      TIMED(RELRES_T_THERMO, launch_thermo(c, sp, k));
    }
  }
  c->cur_step = 0;
  return RELRES_OK;
}

// Instantiated graph for this block (re-captured when an input changed).
static relres_status step_graph(relres_ctx* c, const StepParams& sp, double* d_vel, int blk, int done) {
  const int phase = sp.thermo_every > 0 ? done % sp.thermo_every : 0;
  const int t_phase = done % c->timing_every;
  for (size_t k = 0; k < c->sgs.size(); ++k) {
    const relres_ctx::StepGraph& g = c->sgs[k];
    if (g.valid && g.blk == blk && g.ev_phase == phase && g.thermo_every == sp.thermo_every &&
        g.t_mask == c->timing_mask && g.t_every == c->timing_every && g.t_phase == t_phase &&
        g.timing == int(c->timing) && g.pair_cfg == c->pair_cfg && g.dt == sp.dt && g.t_target == sp.t_target &&
        g.tau == sp.tau && g.n_f == sp.n_f && g.kt == sp.kt && g.seed == sp.seed && g.vel == d_vel &&
        g.thermo == sp.thermo && g.gen == c->buf_gen) {
      c->sg_cur = int(k);
      c->sgs[k].last_use = ++c->sg_clock;
      return RELRES_OK;
    }
  }
  // a free slot: graphs of reallocated buffers first, else the least recently used
  int slot = -1;
  for (size_t k = 0; k < c->sgs.size() && slot < 0; ++k)
    if (!c->sgs[k].valid || c->sgs[k].gen != c->buf_gen) slot = int(k);
  if (slot < 0 && int(c->sgs.size()) < relres_ctx::kMaxStepGraphs) {
    c->sgs.emplace_back();
    slot = int(c->sgs.size()) - 1;
  }
  if (slot < 0) {
    slot = 0;
    for (size_t k = 1; k < c->sgs.size(); ++k)
      if (c->sgs[k].last_use < c->sgs[slot].last_use) slot = int(k);
  }
  c->sg_cur = -1;
  drop_one_graph(c->sgs[slot]);
  relres_ctx::StepGraph& g = c->sgs[slot];
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (!c->body_stream) CK(cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking));
  if (c->timing) {
    g.events.resize(size_t(blk) * 2 * RELRES_T_NCLASS);
    for (cudaEvent_t& e : g.events) CK(cudaEventCreate(&e));
  }
  const long long n0 = c->n_launches;
  const cudaStream_t main = c->stream;
  c->stream = c->cap_stream;
  if (c->timing) {
    c->cap_marks = &g.marks;
    c->cap_events = &g.events;
    c->cap_used = 0;
  }
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  relres_status s = e == cudaSuccess ? record_block(c, sp, d_vel, blk, done, true) : RELRES_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->stream, &graph) : e;
  c->stream = main;
  c->cap_marks = nullptr;
  c->cap_events = nullptr;
  const long long captured = c->n_launches - n0;
  c->n_launches = n0;
  if (s == RELRES_OK && e2 != cudaSuccess) s = fail(c, RELRES_ERR_CUDA, cudaGetErrorString(e2));
  if (s == RELRES_OK) {
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e != cudaSuccess) s = fail(c, RELRES_ERR_CUDA, cudaGetErrorString(e));
  }
  if (graph) cudaGraphDestroy(graph);
  if (s != RELRES_OK) {
    drop_one_graph(g);
    return s;
  }
  // kernels: per step the rebuild body holds kRebuildKernels (binning stages +
  // lists), the pruning body 1, and the decide kernel sits in the parent
  g.k_body = kRebuildKernels;
  g.k_prune = (c->prune_on && !pairs_prune(c)) ? 1 : 0;
  g.k_parent = captured - (g.k_body + g.k_prune) * blk;
  g.valid = true;
  g.blk = blk;
  g.ev_phase = phase;
  g.thermo_every = sp.thermo_every;
  g.timing = int(c->timing);
  g.pair_cfg = c->pair_cfg;
  g.t_mask = c->timing_mask;
  g.t_every = c->timing_every;
  g.t_phase = t_phase;
  g.dt = sp.dt;
  g.t_target = sp.t_target;
  g.tau = sp.tau;
  g.n_f = sp.n_f;
  g.kt = sp.kt;
  g.seed = sp.seed;
  g.vel = d_vel;
  g.thermo = sp.thermo;
  g.gen = c->buf_gen;
  g.last_use = ++c->sg_clock;
  c->sg_cur = slot;
  return RELRES_OK;
}

relres_status relres_set_graphs(relres_ctx* c, int enable) {
  if (!c) return RELRES_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  drop_step_graph(c);
  c->use_graphs = enable != 0;
  return RELRES_OK;
}

relres_status relres_set_params(relres_ctx* c, const relres_params* p) {
  if (!c || !p) return RELRES_ERR_ARG;
  std::vector<PairRecord> recs;
  const std::string e = build_pair_records(p, &recs);
  if (!e.empty()) return fail(c, RELRES_ERR_ARG, e.c_str());
  if (p->n_types != c->n_types || p->mixing != c->prm.mixing || p->precision != c->prm.precision ||
      p->shift != c->prm.shift || p->skin != c->prm.skin)
    return fail(c, RELRES_ERR_ARG, "relres_set_params: n_types, mixing, precision, shift and skin must not change");
  for (int t = 0; t < c->n_types; ++t)
    if (p->is_hybrid[t] != c->is_hybrid[t]) return fail(c, RELRES_ERR_ARG, "relres_set_params: is_hybrid changed");
  for (size_t k = 0; k < recs.size(); ++k) {
    const PairRecord &a = recs[k], &b = c->recs[k];
    if (a.rsm != b.rsm || a.rsp != b.rsp || a.rcm != b.rcm || a.rcp != b.rcp ||
        (a.eps_cg > 0.0) != (b.eps_cg > 0.0))
      return fail(c, RELRES_ERR_ARG, "relres_set_params: radii and the set of CG pairs must not change");
  }
  CK(cudaStreamSynchronize(c->stream));
  c->recs = recs;
  c->eps_fg.assign(p->eps_fg, p->eps_fg + p->n_types);
  c->sig_fg.assign(p->sig_fg, p->sig_fg + p->n_types);
  build_kernel_tables(c->recs, &c->tab_f, &c->tab_d);
  build_basis_tables(c->recs, p->shift, &c->basis_f, &c->basis_d);
  if (c->fp64) {
    CK(cudaMemcpy(c->d_tab, c->tab_d.data(), sizeof(PairTab<double>) * c->tab_d.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_basis, c->basis_d.data(), sizeof(BasisTab<double>) * c->basis_d.size(),
                  cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(c->d_tab, c->tab_f.data(), sizeof(PairTab<float>) * c->tab_f.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_basis, c->basis_f.data(), sizeof(BasisTab<float>) * c->basis_f.size(),
                  cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(c->d_tabd, c->tab_d.data(), sizeof(PairTab<double>) * c->tab_d.size(), cudaMemcpyHostToDevice));
  c->forces_valid = false;
  return RELRES_OK;
}

// dL/d(C12, C6) per record -> dL/d(eps, sig) per record (C12 = 4 eps sig^12,
// C6 = 4 eps sig^6), then the FG ones to the per-type parameters through the
// mixing rule (records (a, b) and (b, a) both depend on type a).
static void chain_params(const relres_ctx* c, const double* gc, double* d_eps_fg, double* d_sig_fg,
                         double* d_eps_cg, double* d_sig_cg) {
  const int nt = c->n_types;
  std::vector<double> de(nt, 0.0), ds(nt, 0.0);
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const int row = a * nt + b;
      const PairRecord& r = c->recs[row];
      const double* g = gc + 4 * row;
      const double sf = r.sig_fg, sc = r.sig_cg;
      const double sf6 = std::pow(sf, 6.0), sc6 = std::pow(sc, 6.0);
      const double e_f = 4.0 * sf6 * sf6 * g[0] + 4.0 * sf6 * g[1];
      const double s_f = 48.0 * r.eps_fg * sf6 * sf6 / sf * g[0] + 24.0 * r.eps_fg * sf6 / sf * g[1];
      if (d_eps_cg) d_eps_cg[row] = r.eps_cg > 0.0 ? 4.0 * sc6 * sc6 * g[2] + 4.0 * sc6 * g[3] : 0.0;
      if (d_sig_cg)
        d_sig_cg[row] =
            r.eps_cg > 0.0 ? 48.0 * r.eps_cg * sc6 * sc6 / sc * g[2] + 24.0 * r.eps_cg * sc6 / sc * g[3] : 0.0;
      const double ea = c->eps_fg[a], eb = c->eps_fg[b], sa = c->sig_fg[a], sb = c->sig_fg[b];
      if (ea > 0.0 && eb > 0.0) {  // eps_ab = sqrt(eps_a eps_b)
        de[a] += e_f * 0.5 * std::sqrt(eb / ea);
        de[b] += e_f * 0.5 * std::sqrt(ea / eb);
      }
      if (c->prm.mixing == RELRES_MIX_LB) {  // sig_ab = (sig_a + sig_b) / 2
        ds[a] += 0.5 * s_f;
        ds[b] += 0.5 * s_f;
      } else {  // sig_ab = sqrt(sig_a sig_b)
        ds[a] += s_f * 0.5 * std::sqrt(sb / sa);
        ds[b] += s_f * 0.5 * std::sqrt(sa / sb);
      }
    }
  if (d_eps_fg) std::copy(de.begin(), de.end(), d_eps_fg);
  if (d_sig_fg) std::copy(ds.begin(), ds.end(), d_sig_fg);
}

relres_status relres_backward(relres_ctx* c, const double* d_pos, const double* d_grad_forces, double grad_energy,
                              double* d_grad_pos, double* grad_c, double* d_eps_fg, double* d_sig_fg,
                              double* d_eps_cg, double* d_sig_cg) {
  if (!c) return RELRES_ERR_ARG;
  if (!c->have_lists) return fail(c, RELRES_ERR_STATE, "relres_build_neighbors first");
  if (!d_pos || !std::isfinite(grad_energy)) return fail(c, RELRES_ERR_ARG, "invalid backward arguments");
  // positions into the device state (lists rebuilt if an atom moved too far)
  c->io_valid = false;
  CK(launch_convert(c, d_pos));
  relres_status s = read_state(c);
  if (s != RELRES_OK) return s;
  if (c->h_state->flags & F_NONFINITE) {
    CK(launch_flags_and(c, ~(unsigned)F_NONFINITE));
    return fail(c, RELRES_ERR_NONFINITE, "non-finite position");
  }
  s = refresh_lists(c);
  if (s != RELRES_OK) return s;
  c->forces_valid = false;
  // gradient buffers (allocated on first use)
  if (c->grad_n != c->n) {
    const size_t vb = c->fp64 ? 24 : 16;
    CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_g_fg), vb * c->n));
    CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_g_cg), vb * std::max(1, c->n_h)));
    CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_gx_fg), vb * c->n));
    CK(dalloc(reinterpret_cast<unsigned char**>(&c->d_gx_cg), vb * c->n));
    CK(dalloc(&c->d_zero_n3, 3 * size_t(c->n)));
    CK(cudaMemsetAsync(c->d_gx_cg, 0, vb * c->n, c->stream));  // ordinary atoms keep zero
    CK(cudaMemsetAsync(c->d_zero_n3, 0, sizeof(double) * 3 * c->n, c->stream));
    c->grad_n = c->n;
  }
  CK(launch_pair_grad(c, d_grad_forces, grad_energy, d_grad_pos));
  std::vector<double> gc(4 * c->recs.size());
  CK(cudaMemcpyAsync(gc.data(), c->d_gc, sizeof(double) * gc.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (grad_c) std::copy(gc.begin(), gc.end(), grad_c);
  chain_params(c, gc.data(), d_eps_fg, d_sig_fg, d_eps_cg, d_sig_cg);
  return RELRES_OK;
}

// State back to the snapshot taken at the start of the current block.
static relres_status rollback_block(relres_ctx* c, double* d_vel) {
  const size_t xb = sizeof(unsigned long long) * 3 * size_t(c->n), vb = sizeof(double) * 3 * size_t(c->n);
  CK(cudaMemcpyAsync(c->d_xfx, c->d_snap_x, xb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(vel_state(c, d_vel), c->d_snap_v, vb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_f_tot, c->d_snap_f, force_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_state, c->d_snap_state, sizeof(DevState), cudaMemcpyDeviceToDevice, c->stream));
  return RELRES_OK;
}

// ---- relres_step in three phases (shared with relres_batch_step)

// Validation, forces at the incoming positions, autotuning, per-call constants.
static relres_status step_begin(relres_ctx* c, int n_steps, double dt_fs, double* d_pos, double* d_vel,
                                double t_target, double tau_fs, uint64_t seed, int thermo_every, double* d_thermo,
                                StepParams* out) {
  if (!c->have_lists) return fail(c, RELRES_ERR_STATE, "relres_build_neighbors first");
  if (n_steps < 0 || !(dt_fs > 0.0) || !std::isfinite(dt_fs) || !d_pos || !d_vel || thermo_every < 0 ||
      (t_target > 0.0 && !(tau_fs > 0.0)))
    return fail(c, RELRES_ERR_ARG, "invalid step arguments");
  StepParams sp{};
  sp.dt = dt_fs;
  sp.t_target = t_target;
  sp.tau = tau_fs;
  sp.n_f = 3.0 * c->n - 3.0;
  sp.kt = 0.5 * sp.n_f * kBoltz * t_target;
  sp.csvr_e = std::exp(-dt_fs / tau_fs);
  sp.seed = seed;
  sp.thermo_every = (d_thermo && thermo_every > 0) ? thermo_every : 0;
  sp.thermo = sp.thermo_every ? d_thermo : nullptr;
  *out = sp;
  if (n_steps == 0) return RELRES_OK;
  if (c->n < 2 && t_target > 0.0) return fail(c, RELRES_ERR_ARG, "the thermostat needs at least 2 atoms");

  // The state at the call's start.  After a relres_step, a call given the
  // arrays that step returned (compared word for word on the device)
  // continues from its end state: the forces are reused and, in FP32 mode
  // with the same time step, so are the velocity state and the last step's
  // thermostat factors (the trajectory is then the bits of one longer call).
  // Otherwise the positions are read and the forces evaluated, and the
  // velocities are read (u = v, a = b = 1).
  const bool cached = c->io_valid && c->forces_valid;
  c->io_valid = false;  // until this call has returned its arrays
  bool dirty = true, keep_u = false;
  relres_status s = RELRES_OK;
  if (cached) {
    const bool try_u = !c->fp64 && dt_fs == c->io_dt;
    CK(launch_flags_and(c, ~(unsigned)(F_DIRTY | F_VDIRTY)));
    CK(launch_check_io(c, d_pos, try_u ? d_vel : nullptr));
    s = read_state(c);
    if (s != RELRES_OK) return s;
    const unsigned fl = c->h_state->flags;
    dirty = (fl & F_DIRTY) != 0;
    keep_u = try_u && !dirty && !(fl & F_VDIRTY);
  }
  if (!keep_u) CK(launch_vel_in(c, d_vel));  // FP32: the float-float velocity state of the call
  CK(launch_call_start(c, !keep_u));
  bool fresh = false;  // host state read after the last device work that changes it
  if (dirty) {
    CK(launch_convert(c, d_pos));
    s = forces_now(c, 0, nullptr, nullptr, nullptr);
    if (s != RELRES_OK) return s;
    fresh = true;
  }
  if (!c->tuned) {
    s = autotune_pairs(c);
    if (s != RELRES_OK) return s;
    fresh = true;
  }
  CK(upload_type_consts(c, dt_fs));
  CK(cudaMemsetAsync(c->d_acc, 0, sizeof(long long) * kNAcc, c->stream));
  // Everything that follows runs on the context stream, after these launches.
  // Without a force evaluation above, the state read at the start is still
  // current for the block accounting (the set-up above changes no count), so
  // no further round trip is needed; after one, read it again.
  return fresh ? read_state(c) : RELRES_OK;
}

// After a block has run: status, timing and launch accounting; on a list
// overflow the state goes back to the block start with larger lists
// (*retry = true); a non-finite force ends the call.
static relres_status block_end(relres_ctx* c, double* d_pos, double* d_vel, double dt_fs, long long builds0,
                               long long prunes0, bool graph, int* retries, bool* retry) {
  *retry = false;
  relres_status s = read_state(c);
  if (s != RELRES_OK) return s;
  s = flush_timing(c);
  if (s != RELRES_OK) return s;
  if (graph) {
    const relres_ctx::StepGraph& sg = c->sgs[c->sg_cur];
    c->n_launches += sg.k_parent + sg.k_body * std::max(0LL, c->h_state->n_builds - builds0) +
                     sg.k_prune * std::max(0LL, (long long)c->h_state->n_prunes - prunes0);
    if (c->timing)
      for (const relres_ctx::Mark& m : sg.marks) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, m.a, m.b));
        c->t_ms[m.cls] += ms;
        c->t_cnt[m.cls] += 1;
      }
  }
  const unsigned fl = c->h_state->flags;
  if (fl & F_BADCELL) return fail(c, RELRES_ERR_CUDA, "cell binning produced an out-of-range index");
  if (fl & (F_OVERFLOW_FG | F_OVERFLOW_CG | F_NONFINITE)) {
    s = rollback_block(c, d_vel);
    if (s != RELRES_OK) return s;
    if (fl & F_NONFINITE) {
      CK(launch_write_back(c, d_pos, d_vel, dt_fs));
      CK(cudaStreamSynchronize(c->stream));
      c->forces_valid = true;
      return fail(c, RELRES_ERR_NONFINITE, "non-finite force during relres_step");
    }
    if (++*retries > 8) {
      CK(launch_write_back(c, d_pos, d_vel, dt_fs));  // the caller's copy of the restored state
      CK(cudaStreamSynchronize(c->stream));
      return fail(c, RELRES_ERR_LIST_OVERFLOW, "repeated list overflow");
    }
    s = read_state(c);
    if (s != RELRES_OK) return s;
    if (fl & F_OVERFLOW_FG) c->cap_fg = round_cap(std::max(c->h_state->max_fg, c->cap_fg) * 1.25 + 8, c->n);
    if (fl & F_OVERFLOW_CG) c->cap_cg = round_cap(std::max(c->h_state->max_cg, c->cap_cg) * 1.25 + 8, c->n_h);
    s = alloc_lists(c);
    if (s != RELRES_OK) return s;
    s = host_rebuild(c);  // lists at the restored positions; F_tot is still theirs
    if (s != RELRES_OK) return s;
    *retry = true;
  }
  return RELRES_OK;
}

// Counters of a completed call; the positions and velocities went back to the
// caller behind its last block, before block_end's status read.
static void step_end(relres_ctx* c, int n_steps, double dt_fs) {
  c->n_steps += n_steps;
  c->step_counter = c->h_state->step;
  c->forces_valid = true;
  c->io_valid = true;
  c->io_dt = dt_fs;
}

// Positions and velocities back to the caller, then the counters (batches).
static relres_status write_back_and_end(relres_ctx* c, int n_steps, double* d_pos, double* d_vel, double dt_fs) {
  CK(launch_write_back(c, d_pos, d_vel, dt_fs));
  relres_status s = read_state(c);
  if (s != RELRES_OK) return s;
  step_end(c, n_steps, dt_fs);
  return RELRES_OK;
}

// ---- batches of independent replicas: one CUDA graph per block of steps
// holds every replica's block on its own branch (fork/join inside one stream
// capture), each with its conditional rebuild nodes and autotuned pair
// launch, so independent systems of any size run concurrently from one graph
// launch and the host checks status once per block for all of them.

struct BatchKey {
  const double* vel;
  double* thermo;
  double t_target, n_f;
  unsigned long long seed;
  long long gen;
  int pair_cfg;
  bool operator==(const BatchKey& o) const {
    return vel == o.vel && thermo == o.thermo && t_target == o.t_target && n_f == o.n_f && seed == o.seed &&
           gen == o.gen && pair_cfg == o.pair_cfg;
  }
};

struct relres_batch {
  std::vector<relres_ctx*> ctx;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> fork;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  cudaGraphExec_t exec = nullptr;
  bool valid = false;
  int blk = 0, phase = 0, thermo_every = 0;
  double dt = 0, tau = 0;
  std::vector<BatchKey> keys;
  std::vector<long long> k_parent;
  bool own_stream = false;
  std::string err;
  // single-launch path: one drift, one pair and one force-sum launch per step
  // for every replica (argument tables in device memory), and the list
  // rebuilds of the replicas that need one in seven launches for all of them
  int mode = -1;                 // relres_batch_set_mode
  std::vector<int> shared;       // replicas in the shared launches of the captured graph
  std::vector<char> is_shared;   // [nrep]
  BatchLaunch bl_pair, bl_drift, bl_sum;
  RebuildBatch rebuild;
  DevState** d_states = nullptr;  // [nrep]
};

static relres_status batch_fail(relres_batch* b, relres_status s, const std::string& m) {
  b->err = m;
  return s;
}

// Replicas can share launches when the kernels' template arguments agree: the
// same precision and force accumulation, and segmented steps.
static bool batch_compatible(const relres_ctx* c, const relres_ctx* ref) {
  return step_segments(c) && c->fp64 == ref->fp64 && c->force_acc == ref->force_acc;
}

// The replicas of the shared launches (relres_batch_set_mode): mode 1 every
// replica (all must be compatible), mode 0 none, mode -1 the compatible
// replicas of at most RELRES_BATCH_SHARED_MAX_ATOMS atoms (at least two).
static relres_status batch_partition(relres_batch* b, std::vector<int>* shared) {
  const int nr = int(b->ctx.size());
  shared->clear();
  if (b->mode == 0) return RELRES_OK;
  if (b->mode == 1) {
    for (int r = 0; r < nr; ++r) {
      if (!batch_compatible(b->ctx[r], b->ctx[0]))
        return batch_fail(b, RELRES_ERR_ARG,
                          "shared launches need replicas of one precision and force accumulation, molecules <= 256 "
                          "atoms");
      shared->push_back(r);
    }
    return RELRES_OK;
  }
  const relres_ctx* ref = nullptr;
  for (int r = 0; r < nr; ++r) {
    relres_ctx* c = b->ctx[r];
    if (c->n > RELRES_BATCH_SHARED_MAX_ATOMS || !step_segments(c)) continue;
    if (!ref) ref = c;
    if (batch_compatible(c, ref)) shared->push_back(r);
  }
  if (shared->size() < 2) shared->clear();
  return RELRES_OK;
}

}  // extern "C"
namespace relres {
cudaError_t upload_batch(BatchLaunch* b, const void* args, size_t bytes, const std::vector<int>& off) {
  if (bytes > b->args_bytes) {
    if (b->d_args) cudaFree(b->d_args);
    b->d_args = nullptr;
    b->args_bytes = 0;
    const cudaError_t e = cudaMalloc(&b->d_args, bytes);
    if (e != cudaSuccess) return e;
    b->args_bytes = bytes;
  }
  if (int(off.size()) > b->n_off) {
    if (b->d_off) cudaFree(b->d_off);
    b->d_off = nullptr;
    b->n_off = 0;
    const cudaError_t e = cudaMalloc(&b->d_off, sizeof(int) * off.size());
    if (e != cudaSuccess) return e;
    b->n_off = int(off.size());
  }
  cudaError_t e = cudaMemcpy(b->d_args, args, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
  return e;
}

void free_batch(BatchLaunch* b) {
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_off) cudaFree(b->d_off);
  *b = BatchLaunch{};
}
}  // namespace relres
extern "C" {

static void batch_drop_graph(relres_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->valid = false;
}

// The shared-launch part of one block of steps, captured on the batch stream
// (tables uploaded beforehand): per replica the rollback snapshot and the
// thermostat draws, then per step the batched drift, the work list of
// replicas whose trigger fired with one conditional node holding the seven
// batched rebuild kernels, the batched pair kernel and the batched force sum.
static relres_status capture_shared(relres_batch* b, const std::vector<relres_ctx*>& cs,
                                    const std::vector<StepParams>& sp, const std::vector<double*>& vel, int blk,
                                    int done) {
  const int ns = int(cs.size());
  const bool fp64 = cs[0]->fp64;
  const int acc = cs[0]->force_acc;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < ns && e == cudaSuccess; ++q) {
    relres_ctx* c = cs[q];
    const size_t xb = sizeof(unsigned long long) * 3 * size_t(c->n), vb = sizeof(double) * 3 * size_t(c->n);
    e = cudaMemcpyAsync(c->d_snap_x, c->d_xfx, xb, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_snap_v, vel_state(c, vel[q]), vb, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_snap_f, c->d_f_tot, force_bytes(c), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_snap_state, c->d_state, sizeof(DevState), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) {
      const cudaStream_t own = c->stream;
      const long long n0 = c->n_launches;  // counted per executed block in k_parent
      c->stream = b->stream;
      e = launch_csvr_draws(c, sp[q], blk);
      c->stream = own;
      c->n_launches = n0;
    }
  }
  relres_status s = RELRES_OK;
  for (int k = 0; k < blk && e == cudaSuccess && s == RELRES_OK; ++k) {
    const bool ev_step = sp[0].thermo_every > 0 && ((done + k + 1) % sp[0].thermo_every) == 0;
    e = launch_drift_batch(b->stream, fp64, ev_step, b->bl_drift, ns);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    cudaGraphConditionalHandle any = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(b->stream, &cst, nullptr, &cg, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&any, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = launch_worklist(b->stream, b->rebuild, b->d_states, ns, any);
    if (e == cudaSuccess) {
      relres_ctx* c0 = cs[0];  // lends its body stream for the capture of the node's body
      const cudaStream_t own = c0->stream;
      c0->stream = b->stream;
      s = add_conditional(c0, any, [b, ns, c0]() { return launch_rebuild_batch(c0->stream, b->rebuild, ns); });
      c0->stream = own;
      if (s != RELRES_OK) b->err = "shared rebuild node (capture): " + c0->err;
    }
    if (e == cudaSuccess && s == RELRES_OK) e = launch_pairs_batch(b->stream, fp64, acc, ev_step, b->bl_pair, ns);
    if (e == cudaSuccess && s == RELRES_OK) e = launch_sum_batch(b->stream, fp64, k, b->bl_sum, ns);
  }
  if (s == RELRES_OK && e != cudaSuccess) s = batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e));
  return s;
}

// Instantiated graph for this block of steps (re-captured when an input
// changed): the replicas of the shared launches on the batch stream, every
// other replica's block on its own branch, all of them concurrently.
static relres_status batch_graph(relres_batch* b, const std::vector<StepParams>& sp, double* const* d_vel, int blk,
                                 int done) {
  const int nr = int(b->ctx.size());
  const int phase = sp[0].thermo_every > 0 ? done % sp[0].thermo_every : 0;
  std::vector<BatchKey> keys(nr);
  for (int r = 0; r < nr; ++r)
    keys[r] = BatchKey{d_vel[r], sp[r].thermo, sp[r].t_target, sp[r].n_f, sp[r].seed, b->ctx[r]->buf_gen,
                       b->ctx[r]->pair_cfg};
  if (b->valid && b->blk == blk && b->phase == phase && b->thermo_every == sp[0].thermo_every &&
      b->dt == sp[0].dt && b->tau == sp[0].tau && b->keys == keys)
    return RELRES_OK;
  batch_drop_graph(b);
  std::vector<int> shared;
  relres_status s = batch_partition(b, &shared);
  if (s != RELRES_OK) return s;
  b->is_shared.assign(nr, 0);
  for (int r : shared) b->is_shared[r] = 1;
  std::vector<relres_ctx*> cs;
  std::vector<StepParams> ssp;
  std::vector<double*> svel;
  for (int r : shared) {
    cs.push_back(b->ctx[r]);
    ssp.push_back(sp[r]);
    svel.push_back(d_vel[r]);
  }
  const int ns = int(cs.size());
  // device tables of the shared launches, uploaded before the capture
  cudaError_t e = cudaSuccess;
  if (ns > 0) {
    e = prepare_pairs_batch(cs, &b->bl_pair);
    if (e == cudaSuccess) e = prepare_drift_batch(cs, ssp, svel.data(), &b->bl_drift);
    if (e == cudaSuccess) e = prepare_sum_batch(cs, ssp, svel.data(), &b->bl_sum);
    if (e == cudaSuccess) e = prepare_rebuild_batch(cs, &b->rebuild);
    if (e == cudaSuccess && !b->d_states) e = cudaMalloc(&b->d_states, sizeof(DevState*) * nr);
    if (e == cudaSuccess) {
      std::vector<DevState*> st(ns);
      for (int q = 0; q < ns; ++q) st[q] = cs[q]->d_state;
      e = cudaMemcpy(b->d_states, st.data(), sizeof(DevState*) * ns, cudaMemcpyHostToDevice);
    }
  }
  // every branch replica (and the shared part) captures its conditional bodies on a stream of its own
  for (int r = 0; r < nr && e == cudaSuccess; ++r)
    if ((!b->is_shared[r] || r == (ns ? shared[0] : -1)) && !b->ctx[r]->body_stream)
      e = cudaStreamCreateWithFlags(&b->ctx[r]->body_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e));
  e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e));
  e = cudaEventRecord(b->ev_fork, b->stream);
  b->k_parent.assign(nr, 0);
  std::vector<int> joins;
  for (int r = 0; r < nr && s == RELRES_OK && e == cudaSuccess; ++r) {
    if (b->is_shared[r]) continue;
    relres_ctx* c = b->ctx[r];
    e = cudaStreamWaitEvent(b->fork[r], b->ev_fork, 0);
    if (e != cudaSuccess) break;
    const cudaStream_t own = c->stream;
    const bool timing = c->timing, pdl = c->use_pdl;
    const long long n0 = c->n_launches;
    c->stream = b->fork[r];
    c->timing = false;  // per-class timing is not recorded in batches
    // no programmatic dependent launches on branches: a kernel waiting for its
    // predecessor would hold SM resources that other branches' kernels can use
    c->use_pdl = false;
    s = record_block(c, sp[r], d_vel[r], blk, done, true);
    c->use_pdl = pdl;
    if (s != RELRES_OK) b->err = "replica " + std::to_string(r) + " (capture): " + c->err;
    const long long kpr = (c->prune_on && !pairs_prune(c)) ? 1 : 0;
    b->k_parent[r] = (c->n_launches - n0) - (kRebuildKernels + kpr) * blk;
    c->stream = own;
    c->timing = timing;
    c->n_launches = n0;
    if (s == RELRES_OK) e = cudaEventRecord(b->ev_join[r], b->fork[r]);
    if (s == RELRES_OK && e == cudaSuccess) joins.push_back(r);
  }
  if (ns > 0 && s == RELRES_OK && e == cudaSuccess) {
    s = capture_shared(b, cs, ssp, svel, blk, done);
    // every shared replica takes part in the step's drift, work-list, pair and force-sum launches
    for (int q = 0; q < ns; ++q) b->k_parent[shared[q]] = 4LL * blk + (ssp[q].t_target > 0.0 ? 1 : 0);
  }
  for (int r : joins)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join[r], 0);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (s == RELRES_OK && e != cudaSuccess) s = batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e));
  if (s == RELRES_OK && e2 != cudaSuccess) s = batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e2));
  if (s == RELRES_OK) {
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) s = batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e));
  }
  if (g) cudaGraphDestroy(g);
  if (s != RELRES_OK) {
    batch_drop_graph(b);
    return s;
  }
  b->shared = shared;
  b->valid = true;
  b->blk = blk;
  b->phase = phase;
  b->thermo_every = sp[0].thermo_every;
  b->dt = sp[0].dt;
  b->tau = sp[0].tau;
  b->keys = keys;
  return RELRES_OK;
}

relres_status relres_batch_create(relres_batch** out, relres_ctx* const* ctxs, int n_ctx, void* cuda_stream) {
  if (!out || !ctxs || n_ctx < 1) return RELRES_ERR_ARG;
  *out = nullptr;
  for (int r = 0; r < n_ctx; ++r) {
    if (!ctxs[r]) return RELRES_ERR_ARG;
    for (int q = 0; q < r; ++q)
      if (ctxs[q] == ctxs[r]) return RELRES_ERR_ARG;
  }
  relres_batch* b = new (std::nothrow) relres_batch();
  if (!b) return RELRES_ERR_NOMEM;
  b->ctx.assign(ctxs, ctxs + n_ctx);
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  b->fork.assign(n_ctx, nullptr);
  b->ev_join.assign(n_ctx, nullptr);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int r = 0; r < n_ctx && e == cudaSuccess; ++r) {
    e = cudaStreamCreateWithFlags(&b->fork[r], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[r], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    relres_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? RELRES_ERR_NOMEM : RELRES_ERR_CUDA;
  }
  *out = b;
  return RELRES_OK;
}

relres_status relres_batch_step(relres_batch* b, int n_steps, double dt_fs, double* const* d_pos,
                                double* const* d_vel, const double* t_target, double tau_fs, const uint64_t* seed,
                                int thermo_every, double* const* d_thermo) {
  if (!b) return RELRES_ERR_ARG;
  if (!d_pos || !d_vel || !t_target || !seed) return batch_fail(b, RELRES_ERR_ARG, "missing per-replica arrays");
  const int nr = int(b->ctx.size());
  std::vector<StepParams> sp(nr);
  for (int r = 0; r < nr; ++r) {
    relres_status s = step_begin(b->ctx[r], n_steps, dt_fs, d_pos[r], d_vel[r], t_target[r], tau_fs, seed[r],
                                 thermo_every, d_thermo ? d_thermo[r] : nullptr, &sp[r]);
    if (s != RELRES_OK)
      return batch_fail(b, s, "replica " + std::to_string(r) + ": " + b->ctx[r]->err);
  }
  if (n_steps == 0) return RELRES_OK;
  int done = 0, retries = 0;
  while (done < n_steps) {
    const int blk = std::min(kBlockSteps, n_steps - done);
    std::vector<long long> builds0(nr), prunes0(nr);
    for (int r = 0; r < nr; ++r) {
      builds0[r] = b->ctx[r]->h_state->n_builds;
      prunes0[r] = (long long)b->ctx[r]->h_state->n_prunes;
    }
    relres_status s = batch_graph(b, sp, d_vel, blk, done);
    if (s != RELRES_OK) return s;
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, RELRES_ERR_CUDA, cudaGetErrorString(e));
    std::vector<unsigned> flags(nr);
    bool overflow = false;
    for (int r = 0; r < nr; ++r) {
      relres_ctx* c = b->ctx[r];
      s = read_state(c);
      if (s != RELRES_OK) return batch_fail(b, s, "replica " + std::to_string(r) + ": " + c->err);
      const long long kpr = (!b->is_shared[r] && c->prune_on && !pairs_prune(c)) ? 1 : 0;
      // a rebuild body of kRebuildKernels kernels runs per rebuild (the shared
      // launches' batched kernels are counted for every replica they rebuild)
      c->n_launches += b->k_parent[r] + kRebuildKernels * std::max(0LL, c->h_state->n_builds - builds0[r]) +
                       kpr * std::max(0LL, (long long)c->h_state->n_prunes - prunes0[r]);
      flags[r] = c->h_state->flags;
      if (flags[r] & F_BADCELL)
        return batch_fail(b, RELRES_ERR_CUDA, "replica " + std::to_string(r) + ": out-of-range cell index");
      if (flags[r] & F_NONFINITE) {
        for (int q = 0; q < nr; ++q) rollback_block(b->ctx[q], d_vel[q]);
        for (int q = 0; q < nr; ++q) write_back_and_end(b->ctx[q], 0, d_pos[q], d_vel[q], dt_fs);
        return batch_fail(b, RELRES_ERR_NONFINITE, "replica " + std::to_string(r) + ": non-finite force");
      }
      overflow |= (flags[r] & (F_OVERFLOW_FG | F_OVERFLOW_CG)) != 0;
    }
    if (overflow) {  // every replica back to the block start; larger lists where they overflowed
      if (++retries > 8) return batch_fail(b, RELRES_ERR_LIST_OVERFLOW, "repeated list overflow");
      for (int r = 0; r < nr; ++r) {
        relres_ctx* c = b->ctx[r];
        s = rollback_block(c, d_vel[r]);
        if (s == RELRES_OK) s = read_state(c);
        if (s == RELRES_OK && (flags[r] & (F_OVERFLOW_FG | F_OVERFLOW_CG))) {
          if (flags[r] & F_OVERFLOW_FG) c->cap_fg = round_cap(std::max(c->h_state->max_fg, c->cap_fg) * 1.25 + 8, c->n);
          if (flags[r] & F_OVERFLOW_CG)
            c->cap_cg = round_cap(std::max(c->h_state->max_cg, c->cap_cg) * 1.25 + 8, c->n_h);
          s = alloc_lists(c);
          if (s == RELRES_OK) s = host_rebuild(c);
        }
        if (s != RELRES_OK) return batch_fail(b, s, "replica " + std::to_string(r) + ": " + c->err);
      }
      continue;
    }
    done += blk;
  }
  for (int r = 0; r < nr; ++r) {
    relres_status s = write_back_and_end(b->ctx[r], n_steps, d_pos[r], d_vel[r], dt_fs);
    if (s != RELRES_OK) return batch_fail(b, s, "replica " + std::to_string(r) + ": " + b->ctx[r]->err);
  }
  return RELRES_OK;
}

const char* relres_batch_last_error(relres_batch* b) { return b ? b->err.c_str() : "null batch"; }

relres_status relres_batch_set_mode(relres_batch* b, int mode) {
  if (!b || mode < -1 || mode > 1) return RELRES_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  b->mode = mode;
  return RELRES_OK;
}

relres_status relres_batch_get_info(relres_batch* b, int* n_shared) {
  if (!b || !n_shared) return RELRES_ERR_ARG;
  *n_shared = b->valid ? int(b->shared.size()) : -1;
  return RELRES_OK;
}

void relres_batch_destroy(relres_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  free_batch(&b->bl_pair);
  free_batch(&b->bl_drift);
  free_batch(&b->bl_sum);
  free_rebuild_batch(&b->rebuild);
  if (b->d_states) cudaFree(b->d_states);
  for (cudaStream_t st : b->fork)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->ev_join)
    if (ev) cudaEventDestroy(ev);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

relres_status relres_step(relres_ctx* c, int n_steps, double dt_fs, double* d_pos, double* d_vel,
                          double t_target, double tau_fs, uint64_t seed, int thermo_every,
                          double* d_thermo) {
  if (!c) return RELRES_ERR_ARG;
  StepParams sp{};
  relres_status s = step_begin(c, n_steps, dt_fs, d_pos, d_vel, t_target, tau_fs, seed, thermo_every, d_thermo, &sp);
  if (s != RELRES_OK || n_steps == 0) return s;
  int done = 0, retries = 0;
  while (done < n_steps) {
    const int blk = std::min(kBlockSteps, n_steps - done);
    const long long builds0 = c->h_state->n_builds, prunes0 = (long long)c->h_state->n_prunes;
    if (c->use_graphs) {
      s = step_graph(c, sp, d_vel, blk, done);
      if (s != RELRES_OK) return s;
      CK(cudaGraphLaunch(c->sgs[c->sg_cur].exec, c->stream));
    } else {
      s = record_block(c, sp, d_vel, blk, done, false);
      if (s != RELRES_OK) return s;
    }
    // behind the last block the positions and velocities go back to the
    // caller, so that one status read covers both (a block that fails or is
    // retried restores the state, and the caller's copy is written again)
    if (done + blk == n_steps) CK(launch_write_back(c, d_pos, d_vel, dt_fs));
    bool retry = false;
    s = block_end(c, d_pos, d_vel, dt_fs, builds0, prunes0, c->use_graphs, &retries, &retry);
    if (s != RELRES_OK) return s;
    if (!retry) done += blk;
  }
  step_end(c, n_steps, dt_fs);
  return RELRES_OK;
}

relres_status relres_set_step_counter(relres_ctx* c, long long step) {
  if (!c || step < 0) return RELRES_ERR_ARG;
  relres_status s = read_state(c);
  if (s != RELRES_OK) return s;
  c->h_state->step = (unsigned long long)step;
  CK(cudaMemcpyAsync(&c->d_state->step, &c->h_state->step, sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->step_counter = (unsigned long long)step;
  return RELRES_OK;
}

relres_status relres_get_stats(relres_ctx* c, relres_stats* o) {
  if (!c || !o) return RELRES_ERR_ARG;
  relres_status s = read_state(c);
  if (s != RELRES_OK) return s;
  std::memset(o, 0, sizeof(*o));
  o->n_atoms = c->n;
  o->n_hybrid = c->n_h;
  o->pair_tpa = c->fp64 ? fp64_pair_tpa(c) : kPairConfigs[c->pair_cfg].tpa;
  o->pair_block = c->fp64 ? fp64_pair_block(c) : kPairConfigs[c->pair_cfg].bs;
  o->cap_fg = c->cap_fg;
  o->cap_cg = c->cap_cg;
  o->max_fg = c->h_state->max_fg;
  o->max_cg = c->h_state->max_cg;
  o->mean_fg = c->n ? double(c->h_state->tot_fg) / c->n : 0.0;
  o->mean_cg = c->n_h ? double(c->h_state->tot_cg) / c->n_h : 0.0;
  o->list_radius_fg = c->rlist_fg_cut + c->prm.skin;
  o->list_radius_cg = c->has_cg ? c->rlist_cg_cut + c->skin_cg : 0.0;
  o->skin_cg = c->skin_cg;
  for (int d = 0; d < 3; ++d) {
    o->grid_fg[d] = c->gfg.n[d];
    o->grid_cg[d] = c->gcg.n[d];
  }
  o->n_builds = c->n_builds + c->h_state->n_builds;
  o->n_steps = (long long)c->h_state->step;
  o->has_cg = c->has_cg ? 1 : 0;
  o->n_launches = c->n_launches;
  o->prune_delta = c->prune_on ? c->prune_delta : 0.0;
  o->step_segments = step_segments(c) ? 1 : 0;
  o->n_segments = c->seg_ok ? c->n_seg : 0;
  o->n_segment_protos = c->seg_ok ? c->n_seg_proto : 0;
  o->force_acc = c->force_acc;
  o->n_prunes = (long long)c->h_state->n_prunes;
  if (c->h_state->n_prunes > 0) {
    const double np = double(c->h_state->n_prunes);
    o->mean_fg_pruned = c->n ? double(c->h_state->tot_in_fg) / (np * c->n) : 0.0;
    o->mean_cg_pruned = c->n_h ? double(c->h_state->tot_in_cg) / (np * c->n_h) : 0.0;
  }
  return RELRES_OK;
}

relres_status relres_set_timing_sampled(relres_ctx* c, unsigned class_mask, int every) {
  if (!c || every < 1) return RELRES_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  relres_status s = flush_timing(c);
  if (s != RELRES_OK) return s;
  c->timing = class_mask != 0;
  c->timing_mask = class_mask;
  c->timing_every = every;
  for (int k = 0; k < RELRES_T_NCLASS; ++k) {
    c->t_ms[k] = 0.0;
    c->t_cnt[k] = 0;
  }
  return RELRES_OK;
}

relres_status relres_set_timing(relres_ctx* c, int enable) {
  if (!c) return RELRES_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  relres_status s = flush_timing(c);
  if (s != RELRES_OK) return s;
  c->timing = enable != 0;
  c->timing_mask = ~0u;
  c->timing_every = 1;
  for (int k = 0; k < RELRES_T_NCLASS; ++k) {
    c->t_ms[k] = 0.0;
    c->t_cnt[k] = 0;
  }
  return RELRES_OK;
}

relres_status relres_get_timings(relres_ctx* c, double* ms, long long* counts, int n) {
  if (!c || n < 0) return RELRES_ERR_ARG;
  for (int k = 0; k < n && k < RELRES_T_NCLASS; ++k) {
    if (ms) ms[k] = c->t_ms[k];
    if (counts) counts[k] = c->t_cnt[k];
  }
  for (int k = RELRES_T_NCLASS; k < n; ++k) {
    if (ms) ms[k] = 0.0;
    if (counts) counts[k] = 0;
  }
  return RELRES_OK;
}

const char* relres_last_error(relres_ctx* c) { return c ? c->err.c_str() : "null context"; }

void relres_destroy(relres_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_step_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->body_stream) cudaStreamDestroy(c->body_stream);
  dfree(c->d_tab);
  dfree(c->d_tabd);
  dfree(c->d_cdt);
  dfree(c->d_mass);
  dfree(c->d_type);
  dfree(c->d_excl_off);
  dfree(c->d_excl_idx);
  dfree(c->d_excl_mask);
  dfree(c->d_bonds);
  dfree(c->d_angles);
  dfree(c->d_dihs);
  dfree(c->d_dih_type);
  dfree(c->d_bond_par);
  dfree(c->d_angle_par);
  dfree(c->d_dih_par);
  dfree(c->d_bond_fpar);
  dfree(c->d_angle_fpar);
  dfree(c->d_inc_off);
  dfree(c->d_inc);
  dfree(c->d_vir_dummy);
  for (Grid* g : {&c->gfg, &c->gcg}) {
    dfree(g->d_rank_of);
    dfree(g->d_start);
    dfree(g->d_count);
    dfree(g->d_tile);
  }
  dfree(c->d_xfx);
  dfree(c->d_ref);
  dfree(c->d_ref_p);
  dfree(c->d_cell_fg);
  dfree(c->d_cell_cg);
  dfree(c->d_slot_fg);
  dfree(c->d_slot_cg);
  dfree(c->d_perm_fg);
  dfree(c->d_rank_fg);
  dfree(c->d_perm_cg);
  dfree(c->d_rank_cg);
  dfree(c->d_pos_fg);
  dfree(c->d_pos_cg);
  dfree(c->d_pos_fg64);
  dfree(c->d_pos_cg64);
  dfree(c->d_nbr_fg);
  dfree(c->d_cnt_fg);
  dfree(c->d_nbr_cg);
  dfree(c->d_cnt_cg);
  dfree(c->d_nbr_fg_in);
  dfree(c->d_cnt_fg_in);
  dfree(c->d_nbr_cg_in);
  dfree(c->d_cnt_cg_in);
  dfree(c->d_f_fg);
  dfree(c->d_f_cg);
  dfree(c->d_f_tot);
  dfree(c->d_f_bond);
  dfree(c->d_tf);
  dfree(c->d_seg);
  dfree(c->d_basis);
  dfree(c->d_gc);
  dfree(c->d_g_fg);
  dfree(c->d_g_cg);
  dfree(c->d_gx_fg);
  dfree(c->d_gx_cg);
  dfree(c->d_zero_n3);
  dfree(c->d_acc);
  dfree(c->d_draws);
  dfree(c->d_state);
  dfree(c->d_out_scratch);
  dfree(c->d_snap_x);
  dfree(c->d_snap_v);
  dfree(c->d_uff);
  dfree(c->d_pos_ret);
  dfree(c->d_vel_ret);
  dfree(c->d_cdt_ff);
  dfree(c->d_kec);
  dfree(c->d_snap_f);
  dfree(c->d_snap_state);
  dfree(c->d_dummy);
  dfree(c->d_open);
  if (c->h_state) cudaFreeHost(c->h_state);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
