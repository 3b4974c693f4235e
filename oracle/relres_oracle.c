/*
 * FP64 CPU oracle for RelRes-LJ molecular dynamics.  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this library.  It shares no code with the CUDA path.
 *
 * Plain, slow, obviously correct:
 *   - oracle_u_tilde: the five-region RelRes potential of Eq. 20 (Section 2.5),
 *     evaluated literally for one type pair, with its r-derivative.
 *   - oracle_pair_forces: sum of Eq. 20 over every non-excluded atom pair
 *     (Eq. 3), minimum image in an orthorhombic periodic box, O(N^2), one
 *     full row per atom (F_i sums over all j != i; energy and virial take half
 *     of each ordered pair).
 *   - oracle_u_tilde_d2, oracle_pair_param_grads, oracle_pair_hvp: second
 *     r-derivative of Eq. 20, the gradient of a function of the pair energy
 *     and forces with respect to every record's eps/sig (through the
 *     derivatives of Eq. 17-19), and the Hessian-vector product of the pair
 *     energy -- the differentiable form of the method, by direct
 *     differentiation.
 *   - oracle_bonded: harmonic bonds E = K (r - r0)^2, harmonic angles
 *     E = K (theta - theta0)^2, OPLS dihedrals
 *     E = 1/2 [K1 (1 + cos phi) + K2 (1 - cos 2phi) + K3 (1 + cos 3phi)
 *             + K4 (1 - cos 4phi)] (Section 3.2 names harmonic bonds/angles
 *     and a Fourier dihedral; the K conventions are this project's reading).
 *   - oracle_md: velocity Verlet with an optional CSVR (Bussi-Donadio-
 *     Parrinello, J. Chem. Phys. 126, 014101 (2007)) thermostat.  Random
 *     numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
 *     counter-based generator, Box-Muller normals, Marsaglia-Tsang (2000) gamma
 *     variates.
 *
 * Units: kcal/mol, Angstrom, fs, g/mol (LAMMPS "real").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One type-pair record; field order matches oracle/params.py ROW_FIELDS. */
typedef struct {
  double eps_fg, sig_fg, eps_cg, sig_cg;
  double rsm, rsp, rcm, rcp; /* r_{s-}, r_{s+}, r_{c-}, r_{c+} */
  double g_fg_m[5];          /* f_{s-}^{FG}, Eq. 17 */
  double g_cg_p[5];          /* f_{s+}^{CG}, Eq. 18 */
  double g_cg_m[5];          /* f_{c-}^{CG}, Eq. 17 */
  double gam_cm, gam_sp, gam_sm; /* Gamma_{c-}, Gamma_{s+}, Gamma_{s-}, Eq. 19 */
} oracle_pair;

/* Eq. 11/12 and its derivative. */
static void lj_u(double r, double eps, double sig, double* u, double* du) {
  if (eps == 0.0) { *u = 0.0; *du = 0.0; return; }
  double s6 = pow(sig / r, 6.0);
  double s12 = s6 * s6;
  *u = 4.0 * eps * (s12 - s6);
  *du = 4.0 * eps * (-12.0 * s12 + 6.0 * s6) / r;
}

/* Eq. 16 and its derivative. */
static void poly_u(const double* g, double d, double* f, double* df) {
  *f = g[0] + g[1] * d + g[2] * d * d + g[3] * d * d * d + g[4] * d * d * d * d;
  *df = g[1] + 2.0 * g[2] * d + 3.0 * g[3] * d * d + 4.0 * g[4] * d * d * d;
}

/* Eq. 20, region by region, half-open intervals as printed. */
static void eq20(const oracle_pair* p, double r, double* u, double* du) {
  double f1, d1, f2, d2;
  if (r < p->rsm) {                       /* [0, r_{s-}) */
    lj_u(r, p->eps_fg, p->sig_fg, &f1, &d1);
    *u = f1 - p->gam_sm;
    *du = d1;
  } else if (r < p->rsp) {                /* [r_{s-}, r_{s+}) */
    double g[5];
    for (int m = 0; m < 5; ++m) g[m] = p->g_fg_m[m] + p->g_cg_p[m];
    poly_u(g, r - p->rsm, &f1, &d1);
    *u = f1 - p->gam_sp;
    *du = d1;
  } else if (r < p->rcm) {                /* [r_{s+}, r_{c-}) */
    lj_u(r, p->eps_cg, p->sig_cg, &f2, &d2);
    *u = f2 - p->gam_cm;
    *du = d2;
  } else if (r < p->rcp) {                /* [r_{c-}, r_{c+}) */
    poly_u(p->g_cg_m, r - p->rcm, &f2, &d2);
    *u = f2 - p->gam_cm;
    *du = d2;
  } else {                                /* [r_{c+}, inf) */
    *u = 0.0;
    *du = 0.0;
  }
}

void oracle_u_tilde(const oracle_pair* p, const double* r, long n, double* u, double* du) {
  for (long k = 0; k < n; ++k) eq20(p, r[k], &u[k], &du[k]);
}

static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

static int is_excluded(const int* off, const int* idx, int i, int j) {
  if (!off) return 0;
  for (int k = off[i]; k < off[i + 1]; ++k)
    if (idx[k] == j) return 1;
  return 0;
}

/* ---- derivatives for the differentiable form ------------------------------ */

/* Eq. 11 with its second r-derivative. */
static void lj_u2(double r, double eps, double sig, double* d2u) {
  if (eps == 0.0) { *d2u = 0.0; return; }
  double s6 = pow(sig / r, 6.0);
  double s12 = s6 * s6;
  *d2u = 4.0 * eps * (156.0 * s12 - 42.0 * s6) / (r * r);
}

static double poly_d2(const double* g, double d) {
  return 2.0 * g[2] + 6.0 * g[3] * d + 12.0 * g[4] * d * d;
}

/* Second r-derivative of Eq. 20, region by region. */
static double eq20_d2(const oracle_pair* p, double r) {
  double v;
  if (r < p->rsm) {
    lj_u2(r, p->eps_fg, p->sig_fg, &v);
    return v;
  }
  if (r < p->rsp) {
    double g[5];
    for (int m = 0; m < 5; ++m) g[m] = p->g_fg_m[m] + p->g_cg_p[m];
    return poly_d2(g, r - p->rsm);
  }
  if (r < p->rcm) {
    lj_u2(r, p->eps_cg, p->sig_cg, &v);
    return v;
  }
  if (r < p->rcp) return poly_d2(p->g_cg_m, r - p->rcm);
  return 0.0;
}

void oracle_u_tilde_d2(const oracle_pair* p, const double* r, long n, double* d2u) {
  for (long k = 0; k < n; ++k) d2u[k] = eq20_d2(p, r[k]);
}

/* d/d eps and d/d sig of u(r) and u'(r) of Eq. 11 (k = 0: eps, 1: sig). */
static void lj_dparam(double r, double eps, double sig, int k, double* du, double* dup) {
  double s6 = pow(sig / r, 6.0);
  double s12 = s6 * s6;
  if (k == 0) {
    *du = 4.0 * (s12 - s6);
    *dup = 4.0 * (-12.0 * s12 + 6.0 * s6) / r;
  } else {
    *du = 4.0 * eps * (12.0 * s12 - 6.0 * s6) / sig;
    *dup = 4.0 * eps * (-144.0 * s12 + 36.0 * s6) / (r * sig);
  }
}

/*
 * Derivative of Eq. 20 (value dv[k] and r-derivative dd[k]) with respect to
 * the four parameters of the record (k: eps_fg, sig_fg, eps_cg, sig_cg).
 * dp[k] holds the derivative of every record field with respect to parameter
 * k (oracle/params.py: pair_row_derivs), so polynomial regions differentiate
 * through their coefficients and the LJ regions analytically.
 */
static void eq20_dparam(const oracle_pair* p, const oracle_pair* dp, double r, double* dv, double* dd) {
  for (int k = 0; k < 4; ++k) {
    double a = 0.0, b = 0.0, f, df;
    if (r < p->rsm) {
      if (k < 2 && p->eps_fg != 0.0) lj_dparam(r, p->eps_fg, p->sig_fg, k, &a, &b);
      a -= dp[k].gam_sm;
    } else if (r < p->rsp) {
      double g[5];
      for (int m = 0; m < 5; ++m) g[m] = dp[k].g_fg_m[m] + dp[k].g_cg_p[m];
      poly_u(g, r - p->rsm, &f, &df);
      a = f - dp[k].gam_sp;
      b = df;
    } else if (r < p->rcm) {
      if (k >= 2 && p->eps_cg != 0.0) lj_dparam(r, p->eps_cg, p->sig_cg, k - 2, &a, &b);
      a -= dp[k].gam_cm;
    } else if (r < p->rcp) {
      poly_u(dp[k].g_cg_m, r - p->rcm, &f, &df);
      a = f - dp[k].gam_cm;
      b = df;
    }
    dv[k] = a;
    dd[k] = b;
  }
}

/*
 * Gradient of a scalar L(E, F) of the pair energy E and the pair forces F with
 * respect to the parameters of every record, given gE = dL/dE and gF[i] =
 * dL/dF_i (may be NULL): out[(a*nt + b)*4 + k].  Each ordered pair (i, j)
 * counts half of its energy derivative, and g_i . dF_ij/dparam, in the record
 * of (type i, type j).
 */
int oracle_pair_param_grads(int n, const double* pos, const double* box, const int* type, int nt,
                            const oracle_pair* table, const oracle_pair* dtable, const int* excl_off,
                            const int* excl_idx, const double* gF, double gE, double* out,
                            int n_threads) {
  const int nr = nt * nt * 4;
  for (int q = 0; q < nr; ++q) out[q] = 0.0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel
  {
    double* loc = (double*)calloc((size_t)nr, sizeof(double));
#pragma omp for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        if (j == i || is_excluded(excl_off, excl_idx, i, j)) continue;
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = min_image(pos[3 * i + a] - pos[3 * j + a], box[a]);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const int row = type[i] * nt + type[j];
        const oracle_pair* p = &table[row];
        if (r >= p->rcp) continue;
        double dv[4], dd[4];
        eq20_dparam(p, &dtable[4 * row], r, dv, dd);
        double gr = 0.0; /* g_i . (r_i - r_j)/r */
        if (gF)
          for (int a = 0; a < 3; ++a) gr += gF[3 * i + a] * d[a] / r;
        for (int k = 0; k < 4; ++k) {
          /* F_ij = -u'(r) (r_i - r_j)/r */
          loc[4 * row + k] += 0.5 * gE * dv[k] - dd[k] * gr;
        }
      }
    }
#pragma omp critical
    for (int q = 0; q < nr; ++q) out[q] += loc[q];
    free(loc);
  }
  return 0;
}

/*
 * Hessian-vector product of the pair energy: out_i = sum_j h_ij (v_i - v_j),
 * h_ij = u''(r) rhat rhat^T + (u'(r)/r) (I - rhat rhat^T), rhat = (r_i - r_j)/r.
 * (The pair forces change by -H v along v.)
 */
int oracle_pair_hvp(int n, const double* pos, const double* box, const int* type, int nt,
                    const oracle_pair* table, const int* excl_off, const int* excl_idx, const double* v,
                    double* out, int n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    double o[3] = {0, 0, 0};
    for (int j = 0; j < n; ++j) {
      if (j == i || is_excluded(excl_off, excl_idx, i, j)) continue;
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = min_image(pos[3 * i + a] - pos[3 * j + a], box[a]);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const oracle_pair* p = &table[type[i] * nt + type[j]];
      if (r >= p->rcp) continue;
      double u, du;
      eq20(p, r, &u, &du);
      const double d2u = eq20_d2(p, r);
      double w[3], rw = 0.0;
      for (int a = 0; a < 3; ++a) {
        w[a] = v[3 * i + a] - v[3 * j + a];
        rw += d[a] / r * w[a];
      }
      for (int a = 0; a < 3; ++a) {
        const double ra = d[a] / r;
        o[a] += d2u * rw * ra + du / r * (w[a] - rw * ra);
      }
    }
    for (int a = 0; a < 3; ++a) out[3 * i + a] = o[a];
  }
  return 0;
}


/*
 * Pair forces, energy and virial of Eq. 20 over all non-excluded pairs.
 * pos: n x 3, box: 3 edge lengths, type: n, table: n_types^2 records (a*nt+b),
 * excl_off/excl_idx: CSR exclusion lists (may be NULL).  forces (n x 3) are
 * overwritten.  energy[0] = total pair energy.  virial[6] = xx yy zz xy xz yz
 * of W_ab = sum_{i<j} (r_i - r_j)_a F_ij,b.  Returns 0.
 */
int oracle_pair_forces(int n, const double* pos, const double* box, const int* type,
                       int nt, const oracle_pair* table, const int* excl_off,
                       const int* excl_idx, double* forces, double* energy,
                       double* virial, int n_threads) {
  double e_tot = 0.0, w[6] = {0, 0, 0, 0, 0, 0};
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel
  {
    double e_loc = 0.0, w_loc[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
      double fi[3] = {0, 0, 0};
      for (int j = 0; j < n; ++j) {
        if (j == i || is_excluded(excl_off, excl_idx, i, j)) continue;
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = min_image(pos[3 * i + a] - pos[3 * j + a], box[a]);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double u, du;
        eq20(&table[type[i] * nt + type[j]], r, &u, &du);
        if (u == 0.0 && du == 0.0) continue;
        /* F_ij = -u'(r) * (r_i - r_j) / r : force on i from j. */
        double s = -du / r;
        for (int a = 0; a < 3; ++a) fi[a] += s * d[a];
        e_loc += 0.5 * u;
        w_loc[0] += 0.5 * d[0] * s * d[0];
        w_loc[1] += 0.5 * d[1] * s * d[1];
        w_loc[2] += 0.5 * d[2] * s * d[2];
        w_loc[3] += 0.5 * d[0] * s * d[1];
        w_loc[4] += 0.5 * d[0] * s * d[2];
        w_loc[5] += 0.5 * d[1] * s * d[2];
      }
      for (int a = 0; a < 3; ++a) forces[3 * i + a] = fi[a];
    }
#pragma omp critical
    {
      e_tot += e_loc;
      for (int c = 0; c < 6; ++c) w[c] += w_loc[c];
    }
  }
  if (energy) energy[0] = e_tot;
  if (virial) memcpy(virial, w, sizeof(w));
  return 0;
}

/*
 * The same all-pairs sum restricted to the rows of `rows` (n_rows atoms):
 * forces[3*k..] = F of atom rows[k] from every other non-excluded atom, and
 * energy[k] = half of that atom's pair energies (so that the rows of all atoms
 * would add up to the total).  Used for bounded samples of large systems.
 */
int oracle_pair_forces_rows(int n, const double* pos, const double* box, const int* type, int nt,
                            const oracle_pair* table, const int* excl_off, const int* excl_idx,
                            int n_rows, const int* rows, double* forces, double* energy,
                            int n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < n_rows; ++k) {
    const int i = rows[k];
    double fi[3] = {0, 0, 0}, ei = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i || is_excluded(excl_off, excl_idx, i, j)) continue;
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = min_image(pos[3 * i + a] - pos[3 * j + a], box[a]);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double u, du;
      eq20(&table[type[i] * nt + type[j]], r, &u, &du);
      if (u == 0.0 && du == 0.0) continue;
      double s = -du / r;
      for (int a = 0; a < 3; ++a) fi[a] += s * d[a];
      ei += 0.5 * u;
    }
    for (int a = 0; a < 3; ++a) forces[3 * k + a] = fi[a];
    if (energy) energy[k] = ei;
  }
  return 0;
}

/* ---------------------------------------------------------------- bonded */

static void sub_mi(const double* pos, const double* box, int a, int b, double* d) {
  /* d = r_a - r_b, minimum image */
  for (int c = 0; c < 3; ++c) d[c] = min_image(pos[3 * a + c] - pos[3 * b + c], box[c]);
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * Bonded forces, ADDED to forces (n x 3).  energy[0..2] = bond, angle,
 * dihedral energies (overwritten).  Parameters per term type:
 * bond_k/bond_r0, ang_k/ang_t0 (radians), dih_k[4*t + 0..3] = K1..K4.
 */
int oracle_bonded(int n, const double* pos, const double* box, int nb, const int* bonds,
                  const int* btype, const double* bond_k, const double* bond_r0, int na,
                  const int* angles, const int* atype, const double* ang_k,
                  const double* ang_t0, int nd, const int* dihs, const int* dtype,
                  const double* dih_k, double* forces, double* energy) {
  (void)n;
  double eb = 0.0, ea = 0.0, ed = 0.0;
  for (int t = 0; t < nb; ++t) {
    int i = bonds[2 * t], j = bonds[2 * t + 1];
    double d[3];
    sub_mi(pos, box, i, j, d);
    double r = sqrt(dot3(d, d));
    double k = bond_k[btype[t]], r0 = bond_r0[btype[t]];
    eb += k * (r - r0) * (r - r0);
    double s = -2.0 * k * (r - r0) / r; /* force on i along d */
    for (int c = 0; c < 3; ++c) {
      forces[3 * i + c] += s * d[c];
      forces[3 * j + c] -= s * d[c];
    }
  }
  for (int t = 0; t < na; ++t) {
    int i = angles[3 * t], j = angles[3 * t + 1], l = angles[3 * t + 2];
    double r1[3], r2[3];
    sub_mi(pos, box, i, j, r1); /* r_i - r_j (j is the vertex) */
    sub_mi(pos, box, l, j, r2); /* r_l - r_j */
    double n1 = sqrt(dot3(r1, r1)), n2 = sqrt(dot3(r2, r2));
    double c = dot3(r1, r2) / (n1 * n2);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double k = ang_k[atype[t]], t0 = ang_t0[atype[t]];
    ea += k * (th - t0) * (th - t0);
    double s = sin(th);
    if (s < 1e-12) s = 1e-12;
    double dEdth = 2.0 * k * (th - t0);
    /* F = -dE/dtheta * dtheta/dc * dc/dr = (dE/dtheta / sin) * dc/dr */
    double pref = dEdth / s;
    for (int q = 0; q < 3; ++q) {
      double dc1 = r2[q] / (n1 * n2) - c * r1[q] / (n1 * n1);
      double dc2 = r1[q] / (n1 * n2) - c * r2[q] / (n2 * n2);
      forces[3 * i + q] += pref * dc1;
      forces[3 * l + q] += pref * dc2;
      forces[3 * j + q] -= pref * (dc1 + dc2);
    }
  }
  for (int t = 0; t < nd; ++t) {
    int i = dihs[4 * t], j = dihs[4 * t + 1], k = dihs[4 * t + 2], l = dihs[4 * t + 3];
    double b1[3], b2[3], b3[3], m1[3], m2[3];
    sub_mi(pos, box, j, i, b1);
    sub_mi(pos, box, k, j, b2);
    sub_mi(pos, box, l, k, b3);
    cross3(b1, b2, m1);
    cross3(b2, b3, m2);
    double nb2 = sqrt(dot3(b2, b2));
    double phi = atan2(nb2 * dot3(b1, m2), dot3(m1, m2));
    const double* K = &dih_k[4 * dtype[t]];
    ed += 0.5 * (K[0] * (1.0 + cos(phi)) + K[1] * (1.0 - cos(2.0 * phi)) +
                 K[2] * (1.0 + cos(3.0 * phi)) + K[3] * (1.0 - cos(4.0 * phi)));
    double dEdphi = 0.5 * (-K[0] * sin(phi) + 2.0 * K[1] * sin(2.0 * phi) -
                           3.0 * K[2] * sin(3.0 * phi) + 4.0 * K[3] * sin(4.0 * phi));
    double mm1 = dot3(m1, m1), mm2 = dot3(m2, m2);
    double b12 = dot3(b1, b2), b32 = dot3(b3, b2);
    for (int q = 0; q < 3; ++q) {
      double gi = -nb2 / mm1 * m1[q];
      double gl = nb2 / mm2 * m2[q];
      double gj = nb2 / mm1 * m1[q] + b12 / (mm1 * nb2) * m1[q] + b32 / (mm2 * nb2) * m2[q];
      double gk = -nb2 / mm2 * m2[q] - b12 / (mm1 * nb2) * m1[q] - b32 / (mm2 * nb2) * m2[q];
      forces[3 * i + q] -= dEdphi * gi;
      forces[3 * j + q] -= dEdphi * gj;
      forces[3 * k + q] -= dEdphi * gk;
      forces[3 * l + q] -= dEdphi * gl;
    }
  }
  if (energy) {
    energy[0] = eb;
    energy[1] = ea;
    energy[2] = ed;
  }
  return 0;
}

/* ------------------------------------------------------------ random numbers */

/* splitmix64 output for counter c under key `seed`: the (c+1)-th output of
 * the sequential generator started at state `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform in (0, 1] from the top 53 bits */
static double unif(uint64_t seed, uint64_t* ctr) {
  uint64_t z = oracle_splitmix64(seed, (*ctr)++);
  return ((double)(z >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* Box-Muller, cosine branch only */
static double normal(uint64_t seed, uint64_t* ctr) {
  double u1 = unif(seed, ctr);
  double u2 = unif(seed, ctr);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Marsaglia-Tsang gamma(a, 1), a >= 1 */
static double gamma_mt(double a, uint64_t seed, uint64_t* ctr) {
  double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  for (int it = 0; it < 1000; ++it) {
    double x = normal(seed, ctr);
    double v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = unif(seed, ctr);
    if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
  }
  return d; /* not reached in practice */
}

/*
 * CSVR velocity scale factor for one step (Bussi et al. 2007, Eq. A7):
 * K_new = K + (1-c)(K_t/N_f (R1^2 + S) - K) + 2 R1 sqrt(c (1-c) K K_t / N_f),
 * c = exp(-dt/tau), K_t = N_f kT / 2, S = sum of N_f-1 squared normals
 * = 2 Gamma((N_f-1)/2).  Random draws of step s use counters s*2^20 + k.
 */
double oracle_csvr_alpha(double ke, double ke_target, double n_f, double dt, double tau,
                         uint64_t seed, uint64_t step) {
  uint64_t ctr = step << 20;
  double c = exp(-dt / tau);
  double r1 = normal(seed, &ctr);
  double s = 2.0 * gamma_mt(0.5 * (n_f - 1.0), seed, &ctr);
  double ke_new = ke + (1.0 - c) * (ke_target / n_f * (r1 * r1 + s) - ke) +
                  2.0 * r1 * sqrt(c * (1.0 - c) * ke * ke_target / n_f);
  return sqrt(ke_new / ke);
}

/* ---------------------------------------------------------------- MD */

#define ORACLE_FTM2V 4.184e-4          /* (kcal/mol/A)/(g/mol) -> A/fs^2 */
#define ORACLE_MVV2E (1.0 / 4.184e-4)  /* (g/mol)(A/fs)^2 -> kcal/mol */
#define ORACLE_KB 0.0019872042586408316 /* R / 4184 J/kcal, kcal/mol/K */

typedef struct {
  int nb; const int* bonds; const int* btype; const double* bond_k; const double* bond_r0;
  int na; const int* angles; const int* atype; const double* ang_k; const double* ang_t0;
  int nd; const int* dihs; const int* dtype; const double* dih_k;
} oracle_topo;

static void all_forces(int n, const double* pos, const double* box, const int* type, int nt,
                       const oracle_pair* table, const int* eo, const int* ei,
                       const oracle_topo* tp, double* f, double* e_pair, double* e_bond,
                       double* vir, int nth) {
  oracle_pair_forces(n, pos, box, type, nt, table, eo, ei, f, e_pair, vir, nth);
  double eb[3] = {0, 0, 0};
  oracle_bonded(n, pos, box, tp->nb, tp->bonds, tp->btype, tp->bond_k, tp->bond_r0, tp->na,
                tp->angles, tp->atype, tp->ang_k, tp->ang_t0, tp->nd, tp->dihs, tp->dtype,
                tp->dih_k, f, eb);
  *e_bond = eb[0] + eb[1] + eb[2];
}

static double kinetic(int n, const double* vel, const double* mass) {
  double k = 0.0;
  for (int i = 0; i < n; ++i)
    k += 0.5 * mass[i] * (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                          vel[3 * i + 2] * vel[3 * i + 2]);
  return k * ORACLE_MVV2E;
}

/*
 * n_steps of velocity Verlet (dt in fs), positions wrapped into [0, L) after
 * each drift.  T_target <= 0: NVE.  Otherwise a CSVR rescale after the second
 * half kick, with N_f = 3n - 3 and time constant tau (fs).  thermo (nullable)
 * receives per step: E_pair, E_bonded, KE (after the thermostat).
 */
int oracle_md(int n, double* pos, double* vel, const double* box, const double* mass,
              const int* type, int nt, const oracle_pair* table, const int* eo, const int* ei,
              const oracle_topo* tp, int n_steps, double dt, double t_target, double tau,
              uint64_t seed, uint64_t step0, double* thermo, int nth) {
  double* f = (double*)calloc((size_t)3 * n, sizeof(double));
  if (!f) return 1;
  double ep, eb, vir[6];
  all_forces(n, pos, box, type, nt, table, eo, ei, tp, f, &ep, &eb, vir, nth);
  double n_f = 3.0 * n - 3.0;
  for (int s = 0; s < n_steps; ++s) {
    for (int i = 0; i < n; ++i) {
      double c = 0.5 * dt * ORACLE_FTM2V / mass[i];
      for (int a = 0; a < 3; ++a) {
        vel[3 * i + a] += c * f[3 * i + a];
        double x = pos[3 * i + a] + dt * vel[3 * i + a];
        x -= box[a] * floor(x / box[a]);
        if (x >= box[a]) x -= box[a];
        pos[3 * i + a] = x;
      }
    }
    all_forces(n, pos, box, type, nt, table, eo, ei, tp, f, &ep, &eb, vir, nth);
    for (int i = 0; i < n; ++i) {
      double c = 0.5 * dt * ORACLE_FTM2V / mass[i];
      for (int a = 0; a < 3; ++a) vel[3 * i + a] += c * f[3 * i + a];
    }
    double ke = kinetic(n, vel, mass);
    if (t_target > 0.0) {
      double kt = 0.5 * n_f * ORACLE_KB * t_target;
      double alpha = oracle_csvr_alpha(ke, kt, n_f, dt, tau, seed, step0 + (uint64_t)s);
      for (int q = 0; q < 3 * n; ++q) vel[q] *= alpha;
      ke *= alpha * alpha;
    }
    if (thermo) {
      thermo[3 * s + 0] = ep;
      thermo[3 * s + 1] = eb;
      thermo[3 * s + 2] = ke;
    }
  }
  free(f);
  return 0;
}
