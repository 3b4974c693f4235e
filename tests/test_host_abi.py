"""Host-side checks of the C-ABI library (no GPU calls).

* librelres.so loads and exports every entry point include/relres.h declares.
* relres_prepare_table (the library's own C++ parameter preparation: mixing,
  Eq. 13, Eq. 17/18, Eq. 19) equals the oracle's pair table.
* relres_cg_params reproduces Table 1 through Eq. 13 under geometric mixing.
* Invalid parameters come back as RELRES_ERR_ARG, never a crash.
"""
import os
import re

import numpy as np
import pytest

from oracle import params as P
from paper_2104_10231_gb300 import relres as R
from paper_2104_10231_gb300 import systems as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_10231_gb300.build import build_library

    build_library()
    return R.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "relres.h")).read()
    decl = r"^(?:relres_status|void|const char\s*\*)\s*(relres_[a-z_]+)\s*\("
    return sorted(set(re.findall(decl, src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "relres_step" in names and "relres_compute" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(R.EXPORTED)


def _compare(sysobj, shift=True):
    p = R.params_for(sysobj, shift=shift)
    got = R.relres_prepare_table(p)
    want = P.pair_table(sysobj.eps_fg, sysobj.sig_fg, sysobj.is_hybrid, sysobj.radii,
                        mixing=sysobj.mixing, group_comp=sysobj.group_comp, shift=shift)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("shift", [True, False])
def test_prepare_table_matches_oracle_propane(lib, shift):
    _compare(S.propane(n_mol=8), shift)


def test_prepare_table_matches_oracle_neopentane(lib):
    _compare(S.neopentane(n_mol=27))


def test_prepare_table_matches_oracle_copolymer_types(lib):
    s = S.neopentane(n_mol=8)
    s = s.subset_copy(eps_fg=np.array([0.0914, 0.195, 0.0914, 0.195]),
                      sig_fg=np.array([3.95, 3.75, 3.95, 3.75]),
                      is_hybrid=np.array([0, 0, 1, 1], np.int32),
                      group_comp=np.array([[0, 0, 0, 0], [0, 0, 0, 0], [4, 0, 1, 0], [0, 4, 0, 1]]),
                      mixing="geometric", radii=(5.5, 6.5, 12.0, 14.0))
    _compare(s)


def test_prepare_table_fg_only_limit(lib):
    _compare(S.fg_only(S.neopentane(n_mol=8)))


def test_prepare_table_explicit_cg_and_pair_radii(lib):
    eps = [0.3, 0.2, 0.25]
    sig = [3.9, 3.7, 4.1]
    hyb = [1, 0, 1]
    ecg = np.array([[2.0, 0.0, 1.5], [0.0, 0.0, 0.0], [1.5, 0.0, 1.2]])
    scg = np.array([[4.0, 3.9, 4.2], [3.9, 3.9, 3.9], [4.2, 3.9, 4.3]])
    rp = np.zeros((3, 3, 4))
    for a in range(3):
        for b in range(3):
            rs = np.sqrt([6.0, 6.5, 7.0][a] * [6.0, 6.5, 7.0][b])
            rp[a, b] = (rs - 0.5, rs + 0.5, 13.0, 14.0)
    p = R.make_params(eps, sig, hyb, (6, 7, 13, 14), 2.0, mixing=R.RELRES_MIX_GEOMETRIC,
                      eps_cg=ecg, sig_cg=scg, radii_pair=rp)
    got = R.relres_prepare_table(p)
    want = P.pair_table(eps, sig, hyb, (6, 7, 13, 14), mixing=P.MIX_GEOMETRIC, eps_cg=ecg,
                        sig_cg=scg, radii_pair=rp)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_cg_params_reproduce_table1(lib):
    from tests.test_oracle_params import _load_table1

    for name, sites, ce, cs in _load_table1():
        eps = [x[0] for x in sites]
        sig = [x[1] for x in sites]
        comp = [1] * len(sites)
        # every site its own type: the group is all types once
        e, s = R.relres_cg_params(eps, sig, R.RELRES_MIX_GEOMETRIC, comp, comp) if len(sites) <= 8 else (0, 0)
        assert e == pytest.approx(ce, rel=5e-4), name
        assert s == pytest.approx(cs, rel=5e-4), name


@pytest.mark.parametrize("bad", ["radii", "eps", "cg_ordinary", "ntypes", "mixing"])
def test_invalid_parameters_are_rejected(lib, bad):
    kw = dict(eps_fg=[0.3, 0.2], sig_fg=[3.9, 3.7], is_hybrid=[1, 0], radii=(6, 7, 13, 14),
              skin=2.0, group_comp=[[1, 2], [0, 0]])
    if bad == "radii":
        kw["radii"] = (7, 6, 13, 14)
    elif bad == "eps":
        kw["eps_fg"] = [-0.3, 0.2]
    elif bad == "cg_ordinary":
        kw.pop("group_comp")
        kw["eps_cg"] = [[1.0, 0.5], [0.5, 0.0]]
        kw["sig_cg"] = [[4.0, 4.0], [4.0, 4.0]]
    elif bad == "ntypes":
        kw["eps_fg"] = [0.1] * 9
        kw["sig_fg"] = [3.9] * 9
        kw["is_hybrid"] = [0] * 9
        kw.pop("group_comp")
    elif bad == "mixing":
        kw["mixing"] = 7
    p = R.make_params(**kw)
    with pytest.raises(R.RelresError) as ei:
        R.relres_prepare_table(p)
    assert ei.value.status == 1


def test_null_handles_and_bad_arguments_fail_before_any_cuda_call(lib):
    # every entry point checks its handle and arguments first: these calls
    # return RELRES_ERR_ARG (or a message) on a machine without a GPU
    import ctypes as C

    ERR = 1  # RELRES_ERR_ARG
    n = C.c_longlong(0)
    st = R.relres_stats()
    assert lib.relres_get_list(None, 0, None, None, 0, C.byref(n)) == ERR
    assert lib.relres_set_prune(None, 0.5) == ERR
    assert lib.relres_set_pair_config(None, 0) == ERR
    assert lib.relres_set_graphs(None, 1) == ERR
    assert lib.relres_set_list_caps(None, 8, 8) == ERR
    assert lib.relres_set_timing(None, 1) == ERR
    assert lib.relres_set_timing_sampled(None, 1, 1) == ERR
    assert lib.relres_get_stats(None, C.byref(st)) == ERR
    assert lib.relres_build_neighbors(None, None, None) == ERR
    assert lib.relres_compute(None, None, None, None, None) == ERR
    assert lib.relres_step(None, 1, 1.0, None, None, 0.0, 100.0, 0, 0, None) == ERR
    assert lib.relres_set_step_counter(None, 0) == ERR
    assert lib.relres_backward(None, None, None, 0.0, None, None, None, None, None, None) == ERR
    assert lib.relres_set_topology(None, None) == ERR
    assert lib.relres_set_params(None, None) == ERR
    assert lib.relres_batch_step(None, 1, 1.0, None, None, None, 100.0, None, 0, None) == ERR
    assert lib.relres_measure_rates(None, 0, None, None) == ERR
    assert lib.relres_eval_recip(None, None, None, 4, None) == ERR
    assert lib.relres_eval_recip(None, None, None, -1, None) == ERR
    assert lib.relres_eval_recip(None, None, None, 0, None) == R.RELRES_OK
    assert lib.relres_create(None, None, None) == ERR
    assert lib.relres_last_error(None) == b"null context"
    assert lib.relres_batch_last_error(None) == b"null batch"
    lib.relres_destroy(None)
    lib.relres_batch_destroy(None)


@pytest.mark.parametrize("mixing", [R.RELRES_MIX_LB, R.RELRES_MIX_GEOMETRIC])
def test_chain_cg_grads_matches_oracle(lib, mixing):
    # relres_chain_cg_grads (C++) against the oracle's chain through Eq. 13
    # (pinned by differences of Eq. 13 in test_oracle_grad.py)
    rule = P.MIX_LB if mixing == R.RELRES_MIX_LB else P.MIX_GEOMETRIC
    rng = np.random.default_rng(2)
    for s in (S.neopentane(n_mol=250, seed=21), S.propane(), S.block_copolymer(n_chain=4)):
        nt = s.n_types
        gec, gsc = rng.normal(size=(nt, nt)), rng.normal(size=(nt, nt))
        gef, gsf = rng.normal(size=nt), rng.normal(size=nt)
        p = R.make_params(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, s.skin, mixing=mixing, group_comp=s.group_comp)
        ge, gs = R.relres_chain_cg_grads(p, gec, gsc, gef, gsf)
        oe, os_ = P.chain_cg_eq13(gef, gsf, gec, gsc, s.eps_fg.astype(float), s.sig_fg.astype(float), s.is_hybrid,
                                  s.group_comp, rule)
        assert np.allclose(ge, oe, rtol=1e-13, atol=1e-13 * np.abs(oe).max()), (s.name, ge, oe)
        assert np.allclose(gs, os_, rtol=1e-13, atol=1e-13 * np.abs(os_).max()), (s.name, gs, os_)


def test_chain_cg_grads_rejects_bad_input(lib):
    s = S.propane()
    nt = s.n_types
    g2, g1 = np.ones((nt, nt)), np.zeros(nt)
    ec, sc = P.cg_table_eq13(s.eps_fg, s.sig_fg, s.is_hybrid, s.group_comp, s.mixing)
    explicit = R.make_params(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, s.skin, eps_cg=ec, sig_cg=sc)
    no_comp = R.make_params(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, s.skin)
    ok = R.make_params(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, s.skin, group_comp=s.group_comp)
    for p, a in ((explicit, g2), (no_comp, g2), (ok, np.full((nt, nt), np.nan))):
        with pytest.raises(R.RelresError) as e:
            R.relres_chain_cg_grads(p, a, g2, g1, g1)
        assert e.value.status == 1  # RELRES_ERR_ARG
    with pytest.raises(ValueError):
        R.relres_chain_cg_grads(ok, g2[:1], g2, g1, g1)
