/*
 * Plain FP64 CPU oracle of the pseudopotential (Shan-Chen) D2Q9 lattice
 * Boltzmann time step of Li, Luo & Li, "Forcing scheme in pseudopotential
 * lattice Boltzmann model for multiphase flows".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no source,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Every operation is written out in the order the paper states it, with no
 * blocking, fusion or reordering:
 *   1. moments       rho = sum_a f_a, u = sum_a f_a e_a / rho   (Sec. III A)
 *   2. potential     psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)) (Eq. 8)
 *                    with p_EOS of Carnahan-Starling            (Eq. 23)
 *   3. force         F = -G psi(x) sum_a w(|e_a|^2) psi(x+e_a) e_a (Eq. 3)
 *                    for every cell before any collision
 *   4. collision     BGK with the chosen forcing scheme         (Eqs. 1, 2,
 *                    9-11, 12-13, 31; Table I)
 *   5. streaming     f_a(x + e_a, t + 1) = f*_a(x, t), periodic  (Eq. 1)
 *
 * Lattice: c = 1, delta_t = 1, c_s^2 = 1/3.  Velocities in the order
 * e0 = (0,0); e1..e4 = (1,0), (0,1), (-1,0), (0,-1); e5..e8 = (1,1), (-1,1),
 * (-1,-1), (1,-1).  Weights 4/9, 1/9, 1/36 (text after Eq. 2).
 * Populations are stored as f[a][y][x] (x fastest), periodic in x and y.
 *
 * Built with -fopenmp (a separate library; the default build has no
 * OpenMP), the loops over cells whose iterations are independent -- moments,
 * potential, force, collision, streaming -- are split over threads.  Each
 * cell's arithmetic is the same, and nothing is summed across cells in
 * those loops, so the result is bit-identical to the single-threaded build.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

static const int ex[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double wq[Q] = {4.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* schemes (same numbering as the public C-ABI, defined here independently) */
enum {
  OR_SC = 0,        /* Shan-Chen velocity shift, Eqs. 9-10            */
  OR_EDM = 1,       /* exact difference method, Eq. 11                */
  OR_IMPROVED = 2,  /* improved scheme, Eq. 31 (sigma = 0: Guo)       */
  OR_NOFORCE = 3,   /* plain BGK, F = 0                               */
  OR_EDM_MOD = 4,   /* EDM with C_e = 1/tau (Sec. III C)              */
  OR_LADD = 5,      /* Ladd, Table I                                  */
  OR_MRT = 6        /* improved forcing in multiple-relaxation-time form
                       (the extension stated at the end of Sec. IV)     */
};

static double cs2(void) { return 1.0 / 3.0; }

int oracle_version(void) { return 1; }

/* Threads used by the cell loops (n > 0 sets it); 1 without OpenMP. */
int oracle_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---- equation of state ------------------------------------------------ */

/* Carnahan-Starling pressure, Eq. 23, with eta = b rho / 4. */
double oracle_p_eos(double rho, double RT, double a, double b) {
  double eta = b * rho / 4.0;
  double num = 1.0 + eta + eta * eta - eta * eta * eta;
  double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
  return rho * RT * num / den - a * rho * rho;
}

/* psi from Eq. 8 with c = 1.  Returns 0 on success, 1 when rho is outside the
 * domain of the potential (rho <= 0, eta >= 1, a negative radicand, or a
 * non-finite value): the oracle never clamps. */
int oracle_psi(double rho, double RT, double a, double b, double G, double *psi) {
  if (!(rho > 0.0) || !isfinite(rho)) return 1;
  if (b * rho / 4.0 >= 1.0) return 1;
  double arg = 2.0 * (oracle_p_eos(rho, RT, a, b) - rho * cs2()) / G;
  if (!(arg >= 0.0) || !isfinite(arg)) return 1;
  *psi = sqrt(arg);
  return 0;
}

/* ---- equilibrium, Eq. 2 ------------------------------------------------ */

void oracle_feq(double rho, double ux, double uy, double *feq) {
  for (int a = 0; a < Q; ++a) {
    double eu = ex[a] * ux + ey[a] * uy;
    double uu = ux * ux + uy * uy;
    /* uu:(e e - c_s^2 I) / (2 c_s^4) = ((e.u)^2 - c_s^2 u.u) / (2 c_s^4) */
    feq[a] = wq[a] * rho *
             (1.0 + eu / cs2() + (eu * eu - cs2() * uu) / (2.0 * cs2() * cs2()));
  }
}

/* ---- step 1: moments --------------------------------------------------- */

void oracle_moments(int nx, int ny, const double *f, double *rho, double *ux,
                    double *uy) {
  int n = nx * ny;
#pragma omp parallel for schedule(static)
  for (int c = 0; c < n; ++c) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; ++a) {
      double fa = f[(size_t)a * n + c];
      r += fa;
      jx += fa * ex[a];
      jy += fa * ey[a];
    }
    rho[c] = r;
    ux[c] = jx / r;
    uy[c] = jy / r;
  }
}

/* ---- step 2: psi field ------------------------------------------------- */

int oracle_psi_field(int nx, int ny, const double *rho, double RT, double a,
                     double b, double G, double *psi) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int c = 0; c < nx * ny; ++c)
    bad |= oracle_psi(rho[c], RT, a, b, G, &psi[c]) != 0;
  return bad;
}

/* ---- step 3: interaction force, Eq. 3 ----------------------------------- */

/* w(|e|^2): w(1) = 1/3 on the axes, w(2) = 1/12 on the diagonals. */
static double w_int(int a) {
  int e2 = ex[a] * ex[a] + ey[a] * ey[a];
  if (e2 == 1) return 1.0 / 3.0;
  if (e2 == 2) return 1.0 / 12.0;
  return 0.0;
}

void oracle_force(int nx, int ny, double G, const double *psi, double *Fx,
                  double *Fy) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double sx = 0.0, sy = 0.0;
      for (int a = 1; a < Q; ++a) {
        int xn = ((x + ex[a]) % nx + nx) % nx;
        int yn = ((y + ey[a]) % ny + ny) % ny;
        double pn = psi[yn * nx + xn];
        sx += w_int(a) * pn * ex[a];
        sy += w_int(a) * pn * ey[a];
      }
      Fx[y * nx + x] = -G * psi[y * nx + x] * sx;
      Fy[y * nx + x] = -G * psi[y * nx + x] * sy;
    }
}

/* ---- step 4: collision at one cell ------------------------------------- */

/* Guo's general forcing term, Eq. 12 with B = B_e F and
 * C = C_e (v F + F v) (Eq. 13 form, arbitrary B_e, C_e and velocity v):
 *   F_a = w_a [ B.e / c_s^2 + C:(e e - c_s^2 I) / (2 c_s^4) ]
 * C:(e e - c_s^2 I) = 2 C_e ((v.e)(F.e) - c_s^2 v.F). */
static double guo_term(int a, double Be, double Ce, double vx, double vy,
                       double Fx, double Fy) {
  double Fe = Fx * ex[a] + Fy * ey[a];
  double ve = vx * ex[a] + vy * ey[a];
  double vF = vx * Fx + vy * Fy;
  double Cee = 2.0 * Ce * (ve * Fe - cs2() * vF);
  return wq[a] * (Be * Fe / cs2() + Cee / (2.0 * cs2() * cs2()));
}

/* Velocities of the improved scheme (Eq. 31, Table I): the actual velocity
 * v = u + F/(2 rho) and v' = v + sigma F / (upsilon psi^2), upsilon = tau - 1/2. */
static void improved_velocities(double rho, double ux, double uy, double Fx, double Fy,
                                double tau, double sigma, double psi, double *vx,
                                double *vy, double *vpx, double *vpy) {
  *vx = ux + Fx / (2.0 * rho);
  *vy = uy + Fy / (2.0 * rho);
  double ups = tau - 0.5;
  *vpx = *vx + sigma * Fx / (ups * psi * psi);
  *vpy = *vy + sigma * Fy / (ups * psi * psi);
}

/* The bracket of the second line of Eq. 31 for direction a:
 * w_a [(e_a - v')/c_s^2 + (e_a.v') e_a / c_s^4] . F */
static double improved_bracket(int a, double vpx, double vpy, double Fx, double Fy) {
  double Fe = Fx * ex[a] + Fy * ey[a];
  double evp = ex[a] * vpx + ey[a] * vpy;
  return wq[a] * (((ex[a] - vpx) * Fx + (ey[a] - vpy) * Fy) / cs2() +
                  evp * Fe / (cs2() * cs2()));
}

/* ---- multiple-relaxation-time form of the improved scheme --------------- */
/* The paper states (end of Sec. IV) that the improved scheme extends to the
 * MRT model without giving the form; this is the reading used here.  The
 * D2Q9 moments are m = M f with the rows (c = e_a, |c|^2 = e.e)
 *   1, -4 + 3|c|^2, 4 - 21|c|^2/2 + 9|c|^4/2, c_x, (-5 + 3|c|^2) c_x,
 *   c_y, (-5 + 3|c|^2) c_y, c_x^2 - c_y^2, c_x c_y
 * (density, energy, energy square, momentum, energy flux, stresses).  The
 * collision relaxes each moment with its own rate towards the moments of
 * f_eq(rho, v) and adds the moments of the improved forcing term with the
 * half-rate factor, m* = m - S (m - M f_eq) + (I - S/2) M Fhat, where
 * Fhat_a = w_a [3 (e_a - v').F + 9 (e_a.v') (e_a.F)] is the bracket of
 * Eq. 31 (so that S = I / tau gives Eq. 31 itself), and f* = M^-1 m*.
 * Rates: stresses 1/tau, energy s_e, energy square s_eps, energy flux s_q
 * (density and momentum: any, their f_eq and forcing moments fix them).
 * A rate <= 0 means 1/tau. */
static double mrt_rates[3] = {0.0, 0.0, 0.0};

void oracle_set_mrt_rates(double s_e, double s_eps, double s_q) {
  mrt_rates[0] = s_e;
  mrt_rates[1] = s_eps;
  mrt_rates[2] = s_q;
}

static void mrt_matrix(double M[Q][Q]) {
  for (int a = 0; a < Q; ++a) {
    double cx = ex[a], cy = ey[a], c2 = cx * cx + cy * cy;
    M[0][a] = 1.0;
    M[1][a] = -4.0 + 3.0 * c2;
    M[2][a] = 4.0 - 10.5 * c2 + 4.5 * c2 * c2;
    M[3][a] = cx;
    M[4][a] = (-5.0 + 3.0 * c2) * cx;
    M[5][a] = cy;
    M[6][a] = (-5.0 + 3.0 * c2) * cy;
    M[7][a] = cx * cx - cy * cy;
    M[8][a] = cx * cy;
  }
}

static int collide_mrt(double tau, double sigma, const double *f, double Fx, double Fy,
                       double psi, double *fout) {
  double M[Q][Q], m[Q];
  mrt_matrix(M);
  for (int k = 0; k < Q; ++k) {
    m[k] = 0.0;
    for (int a = 0; a < Q; ++a) m[k] += M[k][a] * f[a];
  }
  double rho = m[0];                          /* density moment */
  double ux = m[3] / rho, uy = m[5] / rho;    /* momentum moments / rho */
  double vx, vy, vpx, vpy;
  improved_velocities(rho, ux, uy, Fx, Fy, tau, sigma, psi, &vx, &vy, &vpx, &vpy);
  double feq[Q], fhat[Q];
  oracle_feq(rho, vx, vy, feq);
  for (int a = 0; a < Q; ++a) fhat[a] = improved_bracket(a, vpx, vpy, Fx, Fy);
  double sv = 1.0 / tau;
  double se = mrt_rates[0] > 0.0 ? mrt_rates[0] : sv;
  double seps = mrt_rates[1] > 0.0 ? mrt_rates[1] : sv;
  double sq = mrt_rates[2] > 0.0 ? mrt_rates[2] : sv;
  double S[Q] = {sv, se, seps, sv, sq, sv, sq, sv, sv};
  double mstar[Q], norm[Q];
  for (int k = 0; k < Q; ++k) {
    double meq = 0.0, mf = 0.0;
    norm[k] = 0.0;
    for (int a = 0; a < Q; ++a) {
      meq += M[k][a] * feq[a];
      mf += M[k][a] * fhat[a];
      norm[k] += M[k][a] * M[k][a];
    }
    mstar[k] = m[k] - S[k] * (m[k] - meq) + (1.0 - 0.5 * S[k]) * mf;
  }
  /* the rows of M are orthogonal: M^-1 = M^T diag(1 / |row|^2) */
  for (int a = 0; a < Q; ++a) {
    double v = 0.0;
    for (int k = 0; k < Q; ++k) v += M[k][a] * mstar[k] / norm[k];
    fout[a] = v;
  }
  return 0;
}

/* Post-collision populations fout from the pre-collision populations f at one
 * cell, given the interaction force F there and psi there (improved scheme
 * only).  Returns 0, or 1 for an unknown scheme. */
int oracle_collide_cell(int scheme, double tau, double sigma, const double *f,
                        double Fx, double Fy, double psi, double *fout) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int a = 0; a < Q; ++a) {
    rho += f[a];
    jx += f[a] * ex[a];
    jy += f[a] * ey[a];
  }
  double ux = jx / rho, uy = jy / rho; /* u = sum f e / rho */
  double feq[Q], feq2[Q];

  switch (scheme) {
    case OR_SC: { /* Eqs. 9-10: relax towards f_eq(rho, u + tau F / rho) */
      oracle_feq(rho, ux + tau * Fx / rho, uy + tau * Fy / rho, feq);
      for (int a = 0; a < Q; ++a) fout[a] = f[a] - (f[a] - feq[a]) / tau;
      return 0;
    }
    case OR_EDM: { /* Eq. 11: F_a = f_eq(rho, u + du) - f_eq(rho, u), du = F/rho */
      oracle_feq(rho, ux, uy, feq);
      oracle_feq(rho, ux + Fx / rho, uy + Fy / rho, feq2);
      for (int a = 0; a < Q; ++a)
        fout[a] = f[a] - (f[a] - feq[a]) / tau + (feq2[a] - feq[a]);
      return 0;
    }
    case OR_IMPROVED: { /* Eq. 31: Guo with v' = v + sigma F / (upsilon psi^2) */
      double vx, vy, vpx, vpy;
      improved_velocities(rho, ux, uy, Fx, Fy, tau, sigma, psi, &vx, &vy, &vpx, &vpy);
      oracle_feq(rho, vx, vy, feq); /* Guo: f_eq at the actual velocity v */
      for (int a = 0; a < Q; ++a) {
        /* second line of Eq. 31: w (1 - 1/2tau) [(e - v')/c_s^2 + (e.v') e / c_s^4] . F */
        double Fa = (1.0 - 1.0 / (2.0 * tau)) * improved_bracket(a, vpx, vpy, Fx, Fy);
        fout[a] = f[a] - (f[a] - feq[a]) / tau + Fa;
      }
      return 0;
    }
    case OR_NOFORCE: {
      oracle_feq(rho, ux, uy, feq);
      for (int a = 0; a < Q; ++a) fout[a] = f[a] - (f[a] - feq[a]) / tau;
      return 0;
    }
    case OR_EDM_MOD: { /* EDM in Guo form (Eq. 16) with C_e = 1/tau, B_e = 1 */
      double vx = ux + Fx / (2.0 * rho), vy = uy + Fy / (2.0 * rho);
      oracle_feq(rho, ux, uy, feq);
      for (int a = 0; a < Q; ++a)
        fout[a] = f[a] - (f[a] - feq[a]) / tau +
                  guo_term(a, 1.0, 1.0 / tau, vx, vy, Fx, Fy);
      return 0;
    }
    case OR_LADD: { /* Table I: u in f_eq and in F_a, B_e = C_e = 1 */
      oracle_feq(rho, ux, uy, feq);
      for (int a = 0; a < Q; ++a)
        fout[a] = f[a] - (f[a] - feq[a]) / tau +
                  guo_term(a, 1.0, 1.0, ux, uy, Fx, Fy);
      return 0;
    }
    case OR_MRT:
      return collide_mrt(tau, sigma, f, Fx, Fy, psi, fout);
  }
  return 1;
}

/* ---- step 5: streaming -------------------------------------------------- */

void oracle_stream(int nx, int ny, const double *fpost, double *fnew) {
  size_t n = (size_t)nx * ny;
#pragma omp parallel for collapse(2) schedule(static)
  for (int a = 0; a < Q; ++a)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int xd = ((x + ex[a]) % nx + nx) % nx;
        int yd = ((y + ey[a]) % ny + ny) % ny;
        fnew[a * n + (size_t)yd * nx + xd] = fpost[a * n + (size_t)y * nx + x];
      }
}

/* ---- one full step ----------------------------------------------------- */

/* Advance f (in place, [9][ny][nx]) by one time step.  Returns 0, 1 if the
 * density left the domain of psi (divergence; f is left unchanged), or 2 for
 * an invalid argument. */
int oracle_step(int nx, int ny, double *f, int scheme, double tau, double sigma,
                double RT, double a, double b, double G) {
  if (nx < 1 || ny < 1 || !(tau > 0.5)) return 2;
  size_t n = (size_t)nx * ny;
  double *rho = malloc(n * sizeof(double)), *ux = malloc(n * sizeof(double));
  double *uy = malloc(n * sizeof(double)), *psi = malloc(n * sizeof(double));
  double *Fx = malloc(n * sizeof(double)), *Fy = malloc(n * sizeof(double));
  double *fpost = malloc(Q * n * sizeof(double));
  int rc = 0;
  if (!rho || !ux || !uy || !psi || !Fx || !Fy || !fpost) { rc = 2; goto done; }

  oracle_moments(nx, ny, f, rho, ux, uy);
  if (scheme == OR_NOFORCE) { /* F = 0: psi is not needed */
    memset(psi, 0, n * sizeof(double));
    memset(Fx, 0, n * sizeof(double));
    memset(Fy, 0, n * sizeof(double));
  } else {
    if (oracle_psi_field(nx, ny, rho, RT, a, b, G, psi)) { rc = 1; goto done; }
    oracle_force(nx, ny, G, psi, Fx, Fy);
  }
  int bad_scheme = 0;
#pragma omp parallel for schedule(static) reduction(| : bad_scheme)
  for (long long c = 0; c < (long long)n; ++c) {
    double fc[Q], fo[Q];
    for (int q = 0; q < Q; ++q) fc[q] = f[q * n + c];
    if (oracle_collide_cell(scheme, tau, sigma, fc, Fx[c], Fy[c], psi[c], fo)) {
      bad_scheme = 1;
      continue;
    }
    for (int q = 0; q < Q; ++q) fpost[q * n + c] = fo[q];
  }
  if (bad_scheme) { rc = 2; goto done; }
  oracle_stream(nx, ny, fpost, f);
done:
  free(rho); free(ux); free(uy); free(psi); free(Fx); free(Fy); free(fpost);
  return rc;
}

/* steps successive steps; returns the first non-zero step status, and the
 * number of completed steps in *done_steps (may be NULL). */
int oracle_run(int nx, int ny, double *f, int steps, int scheme, double tau,
               double sigma, double RT, double a, double b, double G,
               int *done_steps) {
  int k = 0, rc = 0;
  for (; k < steps; ++k) {
    rc = oracle_step(nx, ny, f, scheme, tau, sigma, RT, a, b, G);
    if (rc) break;
  }
  if (done_steps) *done_steps = k;
  return rc;
}

/* f_a = f_eq(rho, u) at every cell (the initial state). */
void oracle_init_equilibrium(int nx, int ny, const double *rho, const double *ux,
                             const double *uy, double *f) {
  size_t n = (size_t)nx * ny;
  for (size_t c = 0; c < n; ++c) {
    double feq[Q];
    oracle_feq(rho[c], ux ? ux[c] : 0.0, uy ? uy[c] : 0.0, feq);
    for (int a = 0; a < Q; ++a) f[a * n + c] = feq[a];
  }
}

/* A density field at rest: f_a = f_eq(rho, u) with u = -F / (2 rho), where F
 * is the Eq. 3 force of rho itself, so that the actual fluid velocity
 * v = u + F / (2 rho) of Table I vanishes at every cell.  Returns 0, or 1 if
 * psi is undefined somewhere (f is then left unchanged). */
int oracle_init_at_rest(int nx, int ny, const double *rho, double RT, double a,
                        double b, double G, double *f) {
  size_t n = (size_t)nx * ny;
  double *psi = malloc(n * sizeof(double));
  double *Fx = malloc(n * sizeof(double)), *Fy = malloc(n * sizeof(double));
  double *ux = malloc(n * sizeof(double)), *uy = malloc(n * sizeof(double));
  int rc = 0;
  if (!psi || !Fx || !Fy || !ux || !uy) { rc = 2; goto done; }
  if (oracle_psi_field(nx, ny, rho, RT, a, b, G, psi)) { rc = 1; goto done; }
  oracle_force(nx, ny, G, psi, Fx, Fy);
  for (size_t c = 0; c < n; ++c) {
    ux[c] = -Fx[c] / (2.0 * rho[c]);
    uy[c] = -Fy[c] / (2.0 * rho[c]);
  }
  oracle_init_equilibrium(nx, ny, rho, ux, uy, f);
done:
  free(psi); free(Fx); free(Fy); free(ux); free(uy);
  return rc;
}

/* Density and the actual fluid velocity v = u + F / (2 rho) (Table I, every
 * scheme) of the current state; F = 0 when noforce is set.  Returns 0 or 1
 * (psi undefined). */
int oracle_observe(int nx, int ny, const double *f, double RT, double a, double b,
                   double G, int noforce, double *rho, double *vx, double *vy) {
  size_t n = (size_t)nx * ny;
  double *ux = malloc(n * sizeof(double)), *uy = malloc(n * sizeof(double));
  double *psi = malloc(n * sizeof(double));
  double *Fx = malloc(n * sizeof(double)), *Fy = malloc(n * sizeof(double));
  int rc = 0;
  oracle_moments(nx, ny, f, rho, ux, uy);
  if (noforce) {
    memset(Fx, 0, n * sizeof(double));
    memset(Fy, 0, n * sizeof(double));
  } else {
    if (oracle_psi_field(nx, ny, rho, RT, a, b, G, psi)) { rc = 1; goto done; }
    oracle_force(nx, ny, G, psi, Fx, Fy);
  }
  for (size_t c = 0; c < n; ++c) {
    if (vx) vx[c] = ux[c] + Fx[c] / (2.0 * rho[c]);
    if (vy) vy[c] = uy[c] + Fy[c] / (2.0 * rho[c]);
  }
done:
  free(ux); free(uy); free(psi); free(Fx); free(Fy);
  return rc;
}

double oracle_mass(int nx, int ny, const double *f) {
  size_t n = (size_t)nx * ny;
  double m = 0.0;
  for (size_t i = 0; i < Q * n; ++i) m += f[i];
  return m;
}
