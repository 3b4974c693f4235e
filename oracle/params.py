"""Oracle parameter preparation for RelRes-LJ, FP64, restated from Section 2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here follows the paper's notation:

* FG atom types carry ``eps``/``sig``; cross terms by a mixing rule
  (geometric in Section 2.3; Lorentz-Berthelot is the other usual rule).
* The CG pair parameters come from the zero-order multipole sum rule, Eq. 4,
  which for LJ becomes Eq. 13: with A_k = sum_{mu nu} eps_{mu nu} sig_{mu nu}^k
  over the FG sites of the two groups, sig^CG = (A12/A6)^(1/6) and
  eps^CG = A6^2/A12.  Eq. 15 is the per-site form under geometric mixing.
* Eq. 14: a type pair gets eps^CG only when both types are hybrid sites.
* Eq. 16-18: quartic smoothing polynomials f(delta) = sum gamma_m delta^m.
  Eq. 17 switches an interaction off over [r-, r+]; Eq. 18 switches one on.
* Eq. 19: the shift constants Gamma_{c-}, Gamma_{s+}, Gamma_{s-}.

Readings of the paper taken here (each is pinned by a test):

1. Eq. 18's gamma_{4+}: the printed sign of the u'' term is negative.  Solving
   the five conditions of Eq. 8 gives +u''(r+)/(4 dr^2); only that value meets
   f''(dr) = u''(r+), and the printed gamma_{0+} agrees only with it.  We use
   the derived value.
2. A smoothing zone of zero width (r- = r+, allowed in Section 2.5): the zone
   is empty, so only f(0) matters; gamma_3 = gamma_4 = 0 there (Eq. 17/18 would
   divide by zero).
3. ``shift=False`` (the ``pair_modify shift no`` of Section 2.5) sets
   Gamma_{c-} to zero, and Gamma_{s+}, Gamma_{s-} are then formed from Eq. 19
   with that zero, so the energy stays continuous at r_{s-} and r_{s+} and jumps
   only at r_{c+}.  Forces do not depend on any Gamma.
"""
from __future__ import annotations

import math

import numpy as np

MIX_GEOMETRIC = "geometric"
MIX_LB = "lb"

# Row layout of one type-pair record (must match ``oracle_pair`` in
# relres_oracle.c, which is this package's own C part).
ROW_FIELDS = (
    ["eps_fg", "sig_fg", "eps_cg", "sig_cg", "rsm", "rsp", "rcm", "rcp"]
    + [f"g_fg_m{m}" for m in range(5)]
    + [f"g_cg_p{m}" for m in range(5)]
    + [f"g_cg_m{m}" for m in range(5)]
    + ["Gam_cm", "Gam_sp", "Gam_sm"]
)
ROW_LEN = len(ROW_FIELDS)  # 26


def lj(r: float, eps: float, sig: float) -> tuple[float, float, float]:
    """Eq. 11 / Eq. 12: u(r) = 4 eps [(sig/r)^12 - (sig/r)^6] and its first two
    r-derivatives, written out analytically."""
    s6 = (sig / r) ** 6
    s12 = s6 * s6
    u = 4.0 * eps * (s12 - s6)
    du = 4.0 * eps * (-12.0 * s12 + 6.0 * s6) / r
    d2u = 4.0 * eps * (156.0 * s12 - 42.0 * s6) / (r * r)
    return u, du, d2u


def mix_fg(eps, sig, rule: str = MIX_GEOMETRIC):
    """FG cross parameters for every type pair.

    Geometric (Section 2.3): eps_ab = sqrt(eps_a eps_b), sig_ab = sqrt(sig_a sig_b).
    Lorentz-Berthelot: eps geometric, sig arithmetic mean.
    """
    eps = np.asarray(eps, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    E = np.sqrt(np.outer(eps, eps))
    if rule == MIX_GEOMETRIC:
        S = np.sqrt(np.outer(sig, sig))
    elif rule == MIX_LB:
        S = 0.5 * (sig[:, None] + sig[None, :])
    else:
        raise ValueError(f"unknown mixing rule {rule!r}")
    return E, S


def cg_pair_eq13(comp_i, comp_j, E, S) -> tuple[float, float]:
    """Eq. 13: CG pair parameters of groups i and j.

    ``comp_i[t]`` is the number of FG sites of type t in group i (the hybrid
    site included); E, S are the mixed FG parameters.  Returns (eps^CG, sig^CG).
    """
    A6 = 0.0
    A12 = 0.0
    nt = len(comp_i)
    for mu in range(nt):
        for nu in range(nt):
            mult = comp_i[mu] * comp_j[nu]
            if mult == 0:
                continue
            A6 += mult * E[mu, nu] * S[mu, nu] ** 6
            A12 += mult * E[mu, nu] * S[mu, nu] ** 12
    if A6 <= 0.0 or A12 <= 0.0:
        return 0.0, 0.0
    sig_cg = (A12 ** (1.0 / 6.0)) / (A6 ** (1.0 / 6.0))
    eps_cg = A6 * A6 / A12
    return eps_cg, sig_cg


def cg_site_eq15(eps_sites, sig_sites) -> tuple[float, float]:
    """Eq. 15: per-site CG parameters of one group under geometric mixing.

    ``eps_sites``/``sig_sites`` list the FG parameters of every site of the
    group.  Returns (eps_l^CG, sig_l^CG).  Pair values then follow by the
    geometric mean (Section 2.3).
    """
    b6 = sum(math.sqrt(e * s ** 6) for e, s in zip(eps_sites, sig_sites))
    b12 = sum(math.sqrt(e * s ** 12) for e, s in zip(eps_sites, sig_sites))
    sig_l = b12 ** (1.0 / 3.0) / b6 ** (1.0 / 3.0)
    eps_l = b6 ** 4 / b12 ** 2
    return eps_l, sig_l


def cg_table_eq13(eps, sig, is_hybrid, group_comp, rule: str = MIX_GEOMETRIC):
    """CG parameters for every type pair (Eq. 13 for the group pair, then Eq. 14).

    ``group_comp[a]`` (length n_types) is the composition of the group whose
    hybrid site has type a; it is ignored for ordinary types.  Pairs with an
    ordinary type get eps^CG = 0 (Eq. 14) and sig^CG = 0.
    """
    nt = len(eps)
    E, S = mix_fg(eps, sig, rule)
    EC = np.zeros((nt, nt))
    SC = np.zeros((nt, nt))
    for a in range(nt):
        for b in range(nt):
            if is_hybrid[a] and is_hybrid[b]:
                EC[a, b], SC[a, b] = cg_pair_eq13(group_comp[a], group_comp[b], E, S)
    return EC, SC


def switch_off(u: float, du: float, d2u: float, dr: float) -> np.ndarray:
    """Eq. 17: coefficients of f_-(delta), which matches u, u', u'' at delta=0
    and has zero slope and curvature at delta=dr (conditions Eq. 7)."""
    g = np.zeros(5)
    g[0] = u
    g[1] = du
    g[2] = 0.5 * d2u
    if dr > 0.0:
        g[3] = -du / dr ** 2 - 2.0 * d2u / (3.0 * dr)
        g[4] = du / (2.0 * dr ** 3) + d2u / (4.0 * dr ** 2)
    return g


def switch_on(u: float, du: float, d2u: float, dr: float) -> np.ndarray:
    """Eq. 18 (gamma_4 sign as derived from Eq. 8, reading 1 above): f_+(delta)
    has zero slope and curvature at delta=0 and matches u, u', u'' at delta=dr."""
    g = np.zeros(5)
    g[0] = u - 0.5 * du * dr + d2u * dr ** 2 / 12.0
    if dr > 0.0:
        g[3] = du / dr ** 2 - d2u / (3.0 * dr)
        g[4] = -du / (2.0 * dr ** 3) + d2u / (4.0 * dr ** 2)
    return g


def poly(g, delta: float) -> float:
    """Eq. 16: f(delta) = sum_{m=0..4} gamma_m delta^m."""
    return sum(g[m] * delta ** m for m in range(5))


def pair_row(eps_fg, sig_fg, eps_cg, sig_cg, radii, shift: bool = True) -> np.ndarray:
    """One type-pair record: LJ parameters, the four radii, the three smoothing
    polynomials (Eq. 17, Eq. 18, Eq. 17) and the shifts (Eq. 19).

    radii = (r_s-, r_s+, r_c-, r_c+) with r_s- <= r_s+ <= r_c- <= r_c+
    (Section 2.5).
    """
    rsm, rsp, rcm, rcp = (float(x) for x in radii)
    if not (0.0 < rsm <= rsp <= rcm <= rcp):
        raise ValueError("radii must satisfy 0 < r_s- <= r_s+ <= r_c- <= r_c+")
    d_s = rsp - rsm
    d_c = rcp - rcm
    # f_{s-}^{FG}: switches the FG interaction off over [r_s-, r_s+].
    g_fg_m = switch_off(*lj(rsm, eps_fg, sig_fg), d_s) if eps_fg != 0.0 else np.zeros(5)
    if eps_cg != 0.0:
        # f_{s+}^{CG}: switches the CG interaction on over [r_s-, r_s+].
        g_cg_p = switch_on(*lj(rsp, eps_cg, sig_cg), d_s)
        # f_{c-}^{CG}: switches the CG interaction off over [r_c-, r_c+].
        g_cg_m = switch_off(*lj(rcm, eps_cg, sig_cg), d_c)
    else:
        g_cg_p = np.zeros(5)
        g_cg_m = np.zeros(5)
    # Eq. 19 (Eq. 9 written with the polynomials).
    gam_cm = poly(g_cg_m, d_c) if shift else 0.0
    gam_sp = gam_cm + poly(g_fg_m, d_s)
    gam_sm = gam_sp - g_cg_p[0]
    row = np.concatenate((
        [eps_fg, sig_fg, eps_cg, sig_cg, rsm, rsp, rcm, rcp],
        g_fg_m, g_cg_p, g_cg_m,
        [gam_cm, gam_sp, gam_sm],
    )).astype(np.float64)
    assert row.shape == (ROW_LEN,)
    return row


def pair_table(eps, sig, is_hybrid, radii, mixing: str = MIX_GEOMETRIC,
               eps_cg=None, sig_cg=None, group_comp=None, shift: bool = True,
               radii_pair=None) -> np.ndarray:
    """Table of ``pair_row`` records for all n_types x n_types type pairs,
    row-major (a * n_types + b).

    CG parameters come either explicitly (``eps_cg``/``sig_cg`` per type pair,
    like the ``pair_coeff`` of Section 2.5) or from Eq. 13 with ``group_comp``.
    In both cases Eq. 14 zeroes eps^CG of every pair with an ordinary type.
    ``radii_pair`` (n_types x n_types x 4) overrides the global radii per pair.
    """
    nt = len(eps)
    E, S = mix_fg(eps, sig, mixing)
    if eps_cg is None:
        if group_comp is None:
            EC = np.zeros((nt, nt))
            SC = np.zeros((nt, nt))
        else:
            EC, SC = cg_table_eq13(eps, sig, is_hybrid, group_comp, mixing)
    else:
        EC = np.array(eps_cg, dtype=np.float64).reshape(nt, nt)
        SC = np.array(sig_cg, dtype=np.float64).reshape(nt, nt)
    tab = np.zeros((nt * nt, ROW_LEN))
    for a in range(nt):
        for b in range(nt):
            ecg = EC[a, b] if (is_hybrid[a] and is_hybrid[b]) else 0.0
            rr = radii if radii_pair is None else np.asarray(radii_pair)[a, b]
            tab[a * nt + b] = pair_row(E[a, b], S[a, b], ecg, SC[a, b], rr, shift)
    return tab


def row_dict(row) -> dict:
    """Name the fields of one record (for tests and reports)."""
    return {k: float(v) for k, v in zip(ROW_FIELDS, row)}


# ----------------------------------------------------------------- derivatives
#
# Parameter derivatives of Eq. 20 for the differentiable form of the method.
# Every smoothing coefficient of Eq. 17 / Eq. 18 is a fixed linear combination
# of (u, u', u'') at one radius, and Eq. 19 combines the coefficients
# linearly, so the derivative of a record with respect to eps or sig is the
# same construction applied to the derivatives of (u, u', u'') -- written out
# below from Eq. 11 / Eq. 12 directly.

PARAMS = ("eps_fg", "sig_fg", "eps_cg", "sig_cg")


def lj_dparams(r: float, eps: float, sig: float):
    """d/d eps and d/d sig of (u, u', u'') of Eq. 11 at r: two triples."""
    s6 = (sig / r) ** 6
    s12 = s6 * s6
    d_eps = (4.0 * (s12 - s6), 4.0 * (-12.0 * s12 + 6.0 * s6) / r,
             4.0 * (156.0 * s12 - 42.0 * s6) / (r * r))
    # d(s^k)/d sig = k s^k / sig
    d_sig = (4.0 * eps * (12.0 * s12 - 6.0 * s6) / sig,
             4.0 * eps * (-144.0 * s12 + 36.0 * s6) / (r * sig),
             4.0 * eps * (1872.0 * s12 - 252.0 * s6) / (r * r * sig))
    return d_eps, d_sig


def pair_row_derivs(eps_fg, sig_fg, eps_cg, sig_cg, radii, shift: bool = True) -> np.ndarray:
    """(4, ROW_LEN): derivative of every field of ``pair_row`` with respect to
    eps_fg, sig_fg, eps_cg, sig_cg (in that order).  The CG rows are zero
    where eps_cg = 0 (Eq. 14 pairs carry no CG parameters)."""
    rsm, rsp, rcm, rcp = (float(x) for x in radii)
    d_s = rsp - rsm
    d_c = rcp - rcm
    out = np.zeros((4, ROW_LEN))
    zero = np.zeros(5)
    fg_e, fg_s = lj_dparams(rsm, eps_fg, sig_fg)
    if eps_cg != 0.0:
        on_e, on_s = lj_dparams(rsp, eps_cg, sig_cg)
        off_e, off_s = lj_dparams(rcm, eps_cg, sig_cg)
    for k in range(4):
        g_fg_m = zero
        g_cg_p = zero
        g_cg_m = zero
        if k == 0 and eps_fg != 0.0:
            g_fg_m = switch_off(*fg_e, d_s)
        elif k == 1 and eps_fg != 0.0:
            g_fg_m = switch_off(*fg_s, d_s)
        elif k == 2 and eps_cg != 0.0:
            g_cg_p = switch_on(*on_e, d_s)
            g_cg_m = switch_off(*off_e, d_c)
        elif k == 3 and eps_cg != 0.0:
            g_cg_p = switch_on(*on_s, d_s)
            g_cg_m = switch_off(*off_s, d_c)
        gam_cm = poly(g_cg_m, d_c) if shift else 0.0
        gam_sp = gam_cm + poly(g_fg_m, d_s)
        gam_sm = gam_sp - g_cg_p[0]
        head = np.zeros(8)
        head[k] = 1.0
        out[k] = np.concatenate((head, g_fg_m, g_cg_p, g_cg_m, [gam_cm, gam_sp, gam_sm]))
    return out


def table_derivs(eps, sig, is_hybrid, radii, mixing: str = MIX_GEOMETRIC, eps_cg=None, sig_cg=None,
                 group_comp=None, shift: bool = True) -> np.ndarray:
    """(n_types^2, 4, ROW_LEN): ``pair_row_derivs`` of every record of
    ``pair_table`` (same arguments), row-major (a * n_types + b)."""
    tab = pair_table(eps, sig, is_hybrid, radii, mixing, eps_cg, sig_cg, group_comp, shift)
    nt = len(eps)
    out = np.zeros((nt * nt, 4, ROW_LEN))
    for k in range(nt * nt):
        r = tab[k]
        out[k] = pair_row_derivs(r[0], r[1], r[2], r[3], r[4:8], shift)
    return out


def chain_to_types(grad_rows, eps, sig, mixing: str = MIX_GEOMETRIC):
    """Per-record gradients (n_types^2, 4) -- d/d of (eps_fg, sig_fg, eps_cg,
    sig_cg) of each record -- to the per-type FG parameters through the mixing
    rule (both records (a, b) and (b, a) depend on eps_a), and the CG ones
    taken per record (independent leaves).  Returns (d_eps[nt], d_sig[nt],
    d_eps_cg[nt, nt], d_sig_cg[nt, nt])."""
    eps = np.asarray(eps, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    nt = len(eps)
    g = np.asarray(grad_rows, dtype=np.float64).reshape(nt, nt, 4)
    d_eps = np.zeros(nt)
    d_sig = np.zeros(nt)
    for p in range(nt):
        for q in range(nt):
            # eps_pq = sqrt(eps_p eps_q)
            if eps[p] > 0.0 and eps[q] > 0.0:
                d_eps[p] += g[p, q, 0] * 0.5 * math.sqrt(eps[q] / eps[p])
                d_eps[q] += g[p, q, 0] * 0.5 * math.sqrt(eps[p] / eps[q])
            if mixing == MIX_LB:  # sig_pq = (sig_p + sig_q) / 2
                d_sig[p] += 0.5 * g[p, q, 1]
                d_sig[q] += 0.5 * g[p, q, 1]
            else:  # sig_pq = sqrt(sig_p sig_q)
                d_sig[p] += g[p, q, 1] * 0.5 * math.sqrt(sig[q] / sig[p])
                d_sig[q] += g[p, q, 1] * 0.5 * math.sqrt(sig[p] / sig[q])
    return d_eps, d_sig, g[:, :, 2].copy(), g[:, :, 3].copy()


def cg_pair_eq13_vjp(comp_i, comp_j, eps, sig, g_eps_cg: float, g_sig_cg: float,
                     rule: str = MIX_GEOMETRIC):
    """Vector-Jacobian product of Eq. 13 for one group pair: the derivatives of
    g_eps_cg * eps^CG + g_sig_cg * sig^CG with respect to the per-type FG
    parameters (eps[t], sig[t]), through the mixing rule.

    With A_k = sum_{mu nu} n_mu n_nu eps_{mu nu} sig_{mu nu}^k (Eq. 13),
    eps^CG = A6^2 / A12 and sig^CG = (A12 / A6)^(1/6), so
      d eps^CG = (2 A6 / A12) dA6 - (A6^2 / A12^2) dA12,
      d sig^CG = sig^CG / 6 (dA12 / A12 - dA6 / A6),
      dA_k = sum n_mu n_nu (sig_{mu nu}^k d eps_{mu nu} + k eps_{mu nu} sig_{mu nu}^(k-1) d sig_{mu nu}),
    and eps_{mu nu} = sqrt(eps_mu eps_nu), sig_{mu nu} = (sig_mu + sig_nu) / 2 or
    sqrt(sig_mu sig_nu).  A pair with eps_mu = 0 or eps_nu = 0 contributes no eps
    derivative (the convention of ``chain_to_types``).  Zero CG parameters
    (A6 or A12 not positive) depend on nothing.  Returns (d_eps[nt], d_sig[nt])."""
    eps = np.asarray(eps, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    nt = len(eps)
    d_eps = np.zeros(nt)
    d_sig = np.zeros(nt)
    E, S = mix_fg(eps, sig, rule)
    A6 = 0.0
    A12 = 0.0
    for mu in range(nt):
        for nu in range(nt):
            mult = comp_i[mu] * comp_j[nu]
            if mult == 0:
                continue
            A6 += mult * E[mu, nu] * S[mu, nu] ** 6
            A12 += mult * E[mu, nu] * S[mu, nu] ** 12
    if A6 <= 0.0 or A12 <= 0.0:
        return d_eps, d_sig
    sig_cg = (A12 / A6) ** (1.0 / 6.0)
    gA6 = g_eps_cg * 2.0 * A6 / A12 - g_sig_cg * sig_cg / (6.0 * A6)
    gA12 = -g_eps_cg * A6 * A6 / (A12 * A12) + g_sig_cg * sig_cg / (6.0 * A12)
    for mu in range(nt):
        for nu in range(nt):
            mult = comp_i[mu] * comp_j[nu]
            if mult == 0:
                continue
            e, s = E[mu, nu], S[mu, nu]
            g_e = mult * (gA6 * s ** 6 + gA12 * s ** 12)
            g_s = mult * e * (gA6 * 6.0 * s ** 5 + gA12 * 12.0 * s ** 11)
            if eps[mu] > 0.0 and eps[nu] > 0.0:
                d_eps[mu] += g_e * 0.5 * math.sqrt(eps[nu] / eps[mu])
                d_eps[nu] += g_e * 0.5 * math.sqrt(eps[mu] / eps[nu])
            if rule == MIX_LB:
                d_sig[mu] += 0.5 * g_s
                d_sig[nu] += 0.5 * g_s
            else:
                d_sig[mu] += g_s * 0.5 * math.sqrt(sig[nu] / sig[mu])
                d_sig[nu] += g_s * 0.5 * math.sqrt(sig[mu] / sig[nu])
    return d_eps, d_sig


def chain_cg_eq13(d_eps, d_sig, d_eps_cg, d_sig_cg, eps, sig, is_hybrid, group_comp,
                  rule: str = MIX_GEOMETRIC):
    """Total per-type FG gradients when the CG parameters of every hybrid type
    pair follow Eq. 13 from the FG ones: the direct FG gradients (d_eps, d_sig,
    e.g. from ``chain_to_types``) plus, for every record (a, b) with both types
    hybrid (Eq. 14), ``cg_pair_eq13_vjp`` of its CG gradients
    (d_eps_cg[a, b], d_sig_cg[a, b]) with the compositions of the two groups."""
    out_e = np.array(d_eps, dtype=np.float64, copy=True)
    out_s = np.array(d_sig, dtype=np.float64, copy=True)
    nt = len(eps)
    for a in range(nt):
        for b in range(nt):
            if not (is_hybrid[a] and is_hybrid[b]):
                continue
            ge, gs = cg_pair_eq13_vjp(group_comp[a], group_comp[b], eps, sig, d_eps_cg[a][b], d_sig_cg[a][b], rule)
            out_e += ge
            out_s += gs
    return out_e, out_s
