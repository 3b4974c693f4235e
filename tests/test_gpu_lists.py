"""The neighbour lists themselves (Section 2.6: one list for the FG
interactions within r_s+ plus the skin, one over the hybrid atoms for the CG
interactions within r_c+ plus the skin), read back through relres_get_list
and compared with pair sets found by brute force over all atom pairs in FP64.

Index work is held to exact set equality, except for pairs whose distance
lies within TOL of a list radius: the lists decide membership in FP32 from
the 32 high bits of the fixed-point coordinates, the brute force in FP64."""
import numpy as np
import pytest

from paper_2104_10231_gb300 import relres as R
from paper_2104_10231_gb300 import systems as S

pytestmark = pytest.mark.gpu

TOL = 1e-4  # Angstrom
PRUNE_SLACK = 1e-3  # the pruned lists keep pairs within r_cut + delta + this


@pytest.fixture(scope="module")
def torch():
    import torch as T

    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2104_10231_gb300.build import build_library

    build_library()
    R.load()
    return T


def _dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _dist(pos, box, idx):
    """(m, m) minimum-image distances between the atoms idx."""
    p = pos[idx]
    d = p[:, None, :] - p[None, :, :]
    d -= box * np.rint(d / box)
    return np.sqrt((d * d).sum(-1))


def _excluded(s):
    out = set()
    for i in range(s.n_atoms):
        for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]:
            out.add((i, int(j)))
    return out


def _check_list(pairs, pos, box, idx, radius, excl, label):
    """pairs: (n, 2) list entries over the atoms idx; returns the pair set."""
    assert pairs.shape[1] == 2
    if len(pairs):
        assert pairs.min() >= 0, label
    as_set = set(map(tuple, pairs.tolist()))
    assert len(as_set) == len(pairs), f"{label}: duplicate entries"
    assert not any(i == j for i, j in as_set), f"{label}: self pair"
    assert not (as_set & excl), f"{label}: excluded pair listed"
    d = _dist(pos, box, idx)
    loc = {int(a): k for k, a in enumerate(idx)}
    # every listed pair lies within the radius
    for i, j in as_set:
        assert i in loc and j in loc, f"{label}: atom outside the list's atom set"
        assert d[loc[i], loc[j]] < radius + TOL, (label, i, j, d[loc[i], loc[j]], radius)
    # every pair clearly within the radius is listed
    ii, jj = np.nonzero(d < radius - TOL)
    for a, b in zip(idx[ii].tolist(), idx[jj].tolist()):
        if a != b and (a, b) not in excl:
            assert (a, b) in as_set, (label, a, b, radius)
    # full lists: each pair once per owner
    for i, j in as_set:
        if abs(d[loc[i], loc[j]] - radius) > TOL:
            assert (j, i) in as_set, (label, i, j)
    return as_set


def _subsequence_per_owner(inner, outer):
    """The pruned list of each owner keeps the full list's order."""
    by_owner = {}
    for i, j in outer.tolist():
        by_owner.setdefault(i, []).append(j)
    pos_of = {i: {j: k for k, j in enumerate(js)} for i, js in by_owner.items()}
    last = {}
    for i, j in inner.tolist():
        k = pos_of[i][j]
        assert k > last.get(i, -1), (i, j)
        last[i] = k


def _shuffled(s, seed):
    """The same system with its atoms numbered in a random order: each
    molecule's atoms (and so its excluded pairs) lie far apart in atom ids,
    beyond the 15-id reach of the per-atom exclusion masks, so the list build
    searches the exclusion lists instead; bonded terms and exclusions are
    renumbered with the atoms."""
    import dataclasses

    n = s.n_atoms
    perm = np.random.default_rng(seed).permutation(n)  # new atom k is old atom perm[k]
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    off, idx = s.excl
    rows = [np.sort(inv[idx[off[o]:off[o + 1]]]) for o in perm]
    excl_off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    excl_idx = (np.concatenate(rows) if rows else np.zeros(0)).astype(np.int32)
    topo = dict(s.topo)
    for key in ("bonds", "angles", "dihedrals"):
        topo[key] = inv[np.asarray(topo[key], np.int64)].astype(np.int32)
    out = dataclasses.replace(s, name=s.name + "_shuffled", pos=s.pos[perm].copy(), vel=s.vel[perm].copy(),
                              types=s.types[perm].copy(), mol=s.mol[perm].copy(), topo=topo,
                              excl_off=excl_off, excl_idx=excl_idx)
    gaps = [abs(int(j) - k) for k in range(n) for j in excl_idx[excl_off[k]:excl_off[k + 1]]]
    assert max(gaps) > 15
    return out


SYSTEMS = [("propane", lambda: S.propane()),
           ("neopentane shuffled", lambda: _shuffled(S.neopentane(n_mol=500, seed=11), seed=5)),
           ("neopentane", lambda: S.neopentane(n_mol=500, seed=11)),
           ("copolymer", lambda: S.block_copolymer(n_chain=20)),
           ("propane FG only", lambda: S.fg_only(S.propane(), r_inner=9.0, r_outer=10.0))]


@pytest.mark.parametrize("name,make", SYSTEMS, ids=[n for n, _ in SYSTEMS])
@pytest.mark.parametrize("precision", [R.RELRES_PREC_FP32, R.RELRES_PREC_FP64], ids=["fp32", "fp64"])
def test_lists_equal_brute_force_pair_sets(torch, name, make, precision):
    s = make()
    ctx = R.Context(R.params_for(s, precision), R.topology_for(s))
    delta = 0.5
    ctx.set_prune(delta)
    p = _dev(torch, s.pos)
    ctx.build_neighbors(p, s.box)
    torch.cuda.synchronize()
    st = ctx.stats()
    lists = [ctx.get_list(w) for w in range(4)]
    ctx.close()
    excl = _excluded(s)
    all_atoms = np.arange(s.n_atoms)
    hyb = np.nonzero(s.is_hybrid[s.types])[0]
    r_fg = st["list_radius_fg"]
    r_cut_fg = r_fg - s.skin
    fg = _check_list(lists[0], s.pos, s.box, all_atoms, r_fg, excl, "FG")
    rp_fg = min(r_cut_fg + delta + PRUNE_SLACK, r_fg)
    fg_in = _check_list(lists[2], s.pos, s.box, all_atoms, rp_fg, excl, "FG pruned")
    assert fg_in <= fg
    _subsequence_per_owner(lists[2], lists[0])
    assert st["mean_fg"] == pytest.approx(len(lists[0]) / s.n_atoms, rel=1e-12)
    if not st["has_cg"]:
        assert len(lists[1]) == 0 and len(lists[3]) == 0
        return
    r_cg = st["list_radius_cg"]
    r_cut_cg = r_cg - st["skin_cg"]
    cg = _check_list(lists[1], s.pos, s.box, hyb, r_cg, excl, "CG")
    rp_cg = min(r_cut_cg + delta + PRUNE_SLACK, r_cg)
    cg_in = _check_list(lists[3], s.pos, s.box, hyb, rp_cg, excl, "CG pruned")
    assert cg_in <= cg
    _subsequence_per_owner(lists[3], lists[1])
    assert st["n_hybrid"] == len(hyb)
    print(f"{name}: FG {len(fg)} pairs ({len(fg_in)} pruned), CG {len(cg)} ({len(cg_in)} pruned)")


@pytest.mark.parametrize("name,make", SYSTEMS[:3], ids=[n for n, _ in SYSTEMS[:3]])
def test_lists_hold_every_interacting_pair_after_md(torch, name, make):
    # after rebuilds and pruning passes during MD, the lists the pair kernel
    # walks (pruned and full) still hold every pair within the interaction
    # cutoffs at the current positions
    s = make()
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    ctx.set_prune(0.5)
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    ctx.step(400, s.dt, p, v, t_target=s.temperature, tau_fs=100.0, seed=5)
    torch.cuda.synchronize()
    st = ctx.stats()
    lists = [set(map(tuple, ctx.get_list(w).tolist())) for w in range(4)]
    pos = p.cpu().numpy()
    ctx.close()
    assert st["n_prunes"] > 0 and st["n_builds"] > 1, st
    excl = _excluded(s)
    r_cut_fg = st["list_radius_fg"] - s.skin
    d = _dist(pos, s.box, np.arange(s.n_atoms))
    ii, jj = np.nonzero(d < r_cut_fg)
    need = {(a, b) for a, b in zip(ii.tolist(), jj.tolist()) if a != b and (a, b) not in excl}
    assert need <= lists[2] <= lists[0]
    hyb = np.nonzero(s.is_hybrid[s.types])[0]
    r_cut_cg = st["list_radius_cg"] - st["skin_cg"]
    d = _dist(pos, s.box, hyb)
    ii, jj = np.nonzero(d < r_cut_cg)
    need = {(int(hyb[a]), int(hyb[b])) for a, b in zip(ii.tolist(), jj.tolist())
            if a != b and (int(hyb[a]), int(hyb[b])) not in excl}
    assert need <= lists[3] <= lists[1]


def test_list_inspection_errors(torch):
    s = S.propane()
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    with pytest.raises(R.RelresError):
        ctx.get_list(0)  # no lists yet
    ctx.set_prune(0.0)
    ctx.build_neighbors(_dev(torch, s.pos), s.box)
    assert len(ctx.get_list(0)) > 0
    with pytest.raises(R.RelresError):
        ctx.get_list(2)  # pruning is off
    with pytest.raises(R.RelresError):
        ctx.get_list(4)
    ctx.close()
