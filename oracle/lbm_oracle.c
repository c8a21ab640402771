/*
 * FP64 CPU oracle for one time step of the improved three-dimensional
 * colour-gradient MRT lattice Boltzmann model of Wen, Li, Yu and Luo
 * (arXiv:1904.03618).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow restatement that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA sources.
 *
 * Form: the per-colour, literal algorithm, in the paper's order:
 *   moments (Eq. 4, rho^N below Eq. 8, Qbar below Eq. 49),
 *   isotropic gradients (Eq. 49), variable tau_v (Eq. 52),
 *   per colour k: m^k = M f^k, m^{k,eq} = M f^{k,eq} with f^{k,eq} from
 *   Eq. 18 (improved) or Eq. 6 (original), correction C^k (Eq. 45-48),
 *   MRT relaxation in moment space (Eq. 41-42), perturbation Eq. 8 executed
 *   as Lambda * Omega2 (Eq. 53), post-perturbation populations (Eq. 12),
 *   recolouring (Eq. 10-11), streaming (Sec. II.A, below Eq. 13).
 * The perturbation is evaluated in velocity space and the 19x19 matrix work
 * is done densely, on purpose: the CUDA path uses closed forms in moment
 * space, so agreement checks that algebra too.
 *
 * Readings where the paper is silent or inconsistent (each is a parameter or
 * a documented choice here):
 *   - Eq. 18 high-order coefficient: the printed 3/2 gives only half of the
 *     off-diagonal third moments that Eq. 19 and the Appendix require; the
 *     coefficient that reproduces them is 3.  The coefficient is a parameter
 *     (eq18_coef), 3 by default.
 *   - Appendix rows 16-18 as printed disagree with M f^eq; the paper defines
 *     m^eq = M f^eq (Sec. III.B), so m^eq is computed as M f^eq here.
 *   - g^R, g^B of Eq. 52 are not printed: the Grunau / Reis-Phillips
 *     parabolas, continuous with zero slope at +-delta and equal to the
 *     harmonic mean 2 tau_R tau_B / (tau_R + tau_B) at rho^N = 0.
 *   - Body force: Guo forcing in moment space with the same (I - S/2)
 *     factor as the correction term; u carries the F/2 shift; the force on
 *     colour k is (rho_k / rho) F, with F = force + rho * gravity.
 *   - Walls: halfway bounce-back on the two faces of each wall axis; in the
 *     Eq. 49 stencil a neighbour beyond a wall takes the centre-cell value.
 *   - |grad rho^N| < 1e-12: perturbation and recolouring cosine are zero;
 *     cos(phi_0) = 0 for the rest direction.
 *   - BGK variant (collision = 1): Eq. 20 in velocity space with
 *     tau = tau_v of Eq. 52, the correction G^k = M^-1 C^k (the paper obtains
 *     the correction from its moments, C^k = M G^k) and the Guo force term
 *     both under the factor (1 - 1/(2 tau)), and the perturbation of Eq. 8
 *     divided by tau (the treatment that makes the surface tension
 *     independent of tau, of which Eq. 53 is the MRT form).  The paper
 *     states that Eq. 40 reduces to Eq. 20 for Lambda = I / tau; this
 *     branch is written without M, S or Lambda so that the two check each
 *     other.
 *   - Moving plates (wall = 2, Sec. IV.A): Zou-He velocity nodes.  The
 *     first and last layer of the axis lie on plates moving with wall_u;
 *     after streaming, the populations that would enter from beyond a plate
 *     are rebuilt per colour k from the known ones: rho_k from mass and the
 *     plate's normal velocity, the bounce-back of the non-equilibrium part
 *     along the normal, and transverse corrections N_t that make the
 *     colour's momentum exactly rho_k u_w (the D3Q19 form of Hecht and
 *     Harting).  Populations leaving through a plate are dropped.  In the
 *     Eq. 49 stencil a plate acts as a wall.  The plate velocity carries no
 *     forcing shift (the paper's case has no body force).
 *   - Wetting (optional; the paper uses only the neutral wall, theta = 90
 *     degrees): at a fluid cell next to a wall the colour gradient keeps its
 *     magnitude and its direction along the wall but is turned to make the
 *     angle pi - theta with the inward wall normal (theta measured through
 *     the red phase), and this gradient then drives the perturbation and the
 *     recolouring.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lbm_oracle.h"

/* D3Q19 velocities, Eq. 5 (column i of the printed matrix). */
static const int E[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Weights omega_i, stated below Eq. 6. */
static double weight(int i) {
  if (i == 0) return 1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* B_i of the perturbation operator, stated below Eq. 8. */
static double bcoef(int i) {
  if (i == 0) return -1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* phi_i^k of Eq. 13. */
static double phi(int i, double alpha) {
  if (i == 0) return alpha;
  if (i <= 6) return (1.0 - alpha) / 12.0;
  return (1.0 - alpha) / 24.0;
}

/* Index of the opposite direction -e_i. */
static int opposite(int i) {
  for (int j = 0; j < 19; ++j)
    if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2])
      return j;
  return -1;
}

/* Row r of the transformation matrix, Eq. 43, evaluated at velocity e. */
static double moment_row(int r, const int *e) {
  double x = e[0], y = e[1], z = e[2];
  switch (r) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x + y * y + z * z;
    case 5: return 2 * x * x - y * y - z * z;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * y;
    case 11: return x * y * y;
    case 12: return x * x * z;
    case 13: return x * z * z;
    case 14: return y * y * z;
    case 15: return y * z * z;
    case 16: return x * x * y * y;
    case 17: return x * x * z * z;
    case 18: return y * y * z * z;
  }
  return 0.0;
}

void or_matrix_M(double *M) {
  for (int r = 0; r < 19; ++r)
    for (int i = 0; i < 19; ++i) M[r * 19 + i] = moment_row(r, E[i]);
}

/* Gauss-Jordan inversion with partial pivoting (a library-style step). */
int or_matrix_Minv(double *Minv) {
  double a[19][38];
  double M[361];
  or_matrix_M(M);
  for (int r = 0; r < 19; ++r)
    for (int c = 0; c < 38; ++c)
      a[r][c] = c < 19 ? M[r * 19 + c] : (c - 19 == r ? 1.0 : 0.0);
  for (int c = 0; c < 19; ++c) {
    int piv = c;
    for (int r = c + 1; r < 19; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (fabs(a[piv][c]) < 1e-14) return -1;
    if (piv != c)
      for (int k = 0; k < 38; ++k) {
        double t = a[c][k];
        a[c][k] = a[piv][k];
        a[piv][k] = t;
      }
    double d = a[c][c];
    for (int k = 0; k < 38; ++k) a[c][k] /= d;
    for (int r = 0; r < 19; ++r)
      if (r != c) {
        double f = a[r][c];
        if (f != 0.0)
          for (int k = 0; k < 38; ++k) a[r][k] -= f * a[c][k];
      }
  }
  for (int r = 0; r < 19; ++r)
    for (int c = 0; c < 19; ++c) Minv[r * 19 + c] = a[r][19 + c];
  return 0;
}

static void matvec(const double *A, const double *x, double *y) {
  for (int r = 0; r < 19; ++r) {
    double s = 0.0;
    for (int c = 0; c < 19; ++c) s += A[r * 19 + c] * x[c];
    y[r] = s;
  }
}

/* Equilibrium of colour k: Eq. 18 (improved, with the high-order term
   weighted by eq18_coef) or Eq. 6 (original, no high-order term).
   c = 1 throughout (below Eq. 5); (c_s^k)^2 = (1 - alpha_k)/2 (Eq. 13). */
void or_feq(double rho_k, double alpha_k, const double *u, int improved,
            double eq18_coef, double *feq) {
  double cs2 = 0.5 * (1.0 - alpha_k);
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 19; ++i) {
    double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
    double ee = E[i][0] * E[i][0] + E[i][1] * E[i][1] + E[i][2] * E[i][2];
    double bracket = 3.0 * eu + 4.5 * eu * eu - 1.5 * uu;
    if (improved)
      bracket += eq18_coef * eu * (3.0 * cs2 - 1.0) * (3.0 * ee - 5.0);
    feq[i] = rho_k * (phi(i, alpha_k) + weight(i) * bracket);
  }
}

/* Guo forcing term for a force density Fk at velocity u (velocity space):
   F_i = omega_i [ 3 (e_i - u) . Fk + 9 (e_i . u)(e_i . Fk) ]. */
void or_force_guo(const double *Fk, const double *u, double *Fi) {
  for (int i = 0; i < 19; ++i) {
    double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
    double eF = E[i][0] * Fk[0] + E[i][1] * Fk[1] + E[i][2] * Fk[2];
    double uF = u[0] * Fk[0] + u[1] * Fk[1] + u[2] * Fk[2];
    Fi[i] = weight(i) * (3.0 * (eF - uF) + 9.0 * eu * eF);
  }
}

/* Perturbation operator of one colour, Eq. 8, in velocity space. */
void or_perturbation(double A_k, const double *grad, double *om2) {
  double g2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2];
  double g = sqrt(g2);
  for (int i = 0; i < 19; ++i) {
    if (g < OR_GRAD_EPS) {
      om2[i] = 0.0;
      continue;
    }
    double eg = E[i][0] * grad[0] + E[i][1] * grad[1] + E[i][2] * grad[2];
    om2[i] = 0.5 * A_k * g * (weight(i) * eg * eg / g2 - bcoef(i));
  }
}

/* Correction term in moment space, Eq. 45, from (Q_x, Q_y, Q_z). */
void or_correction(const double *Q, double *C) {
  for (int r = 0; r < 19; ++r) C[r] = 0.0;
  C[4] = Q[0] + Q[1] + Q[2];
  C[5] = 2.0 * Q[0] - Q[1] - Q[2];
  C[6] = Q[1] - Q[2];
}

/* Contact-angle rule at a wall-adjacent cell.  wall_side[a] = +1 if the
   cell touches the wall at the low face of axis a (inward normal +e_a),
   -1 at the high face, 0 otherwise.  grad is modified in place. */
void or_wetting(const int *wall_side, double theta_deg, double *grad) {
  double n[3] = {(double)wall_side[0], (double)wall_side[1], (double)wall_side[2]};
  double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  if (nn == 0.0) return;
  for (int a = 0; a < 3; ++a) n[a] /= sqrt(nn);
  double gn = grad[0] * n[0] + grad[1] * n[1] + grad[2] * n[2];
  double t[3], tt = 0.0, g2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    t[a] = grad[a] - gn * n[a];
    tt += t[a] * t[a];
    g2 += grad[a] * grad[a];
  }
  if (tt <= 0.0 || g2 <= 0.0) return;
  double theta = theta_deg * M_PI / 180.0;
  double g = sqrt(g2), tl = sqrt(tt);
  for (int a = 0; a < 3; ++a)
    grad[a] = g * (-cos(theta) * n[a] + sin(theta) * t[a] / tl);
}

/* Relaxation time tau_v of Eq. 52 with the parabolic g^R, g^B. */
double or_tau_v(double rhoN, double tau_R, double tau_B, double delta) {
  double s = 2.0 * tau_R * tau_B / (tau_R + tau_B);
  if (rhoN > delta) return tau_R;
  if (rhoN > 0.0) {
    double a = 2.0 * (tau_R - s) / delta;
    return s + a * rhoN - a / (2.0 * delta) * rhoN * rhoN;
  }
  if (rhoN >= -delta) {
    double b = 2.0 * (s - tau_B) / delta;
    return s + b * rhoN + b / (2.0 * delta) * rhoN * rhoN;
  }
  return tau_B;
}

/* Relaxation matrix diagonal, Eq. 44. */
static void relaxation_diag(const or_params *p, double tau_v, double *s) {
  for (int r = 0; r < 4; ++r) s[r] = 1.0;
  s[4] = 1.0 / p->tau_e;
  for (int r = 5; r < 10; ++r) s[r] = 1.0 / tau_v;
  for (int r = 10; r < 16; ++r) s[r] = 1.0 / p->tau_q;
  for (int r = 16; r < 19; ++r) s[r] = 1.0 / p->tau_pi;
}

/* ---- lattice indexing --------------------------------------------------- */

static long cell_index(const or_params *p, int x, int y, int z) {
  return ((long)z * p->ny + y) * p->nx + x;
}

/* Neighbour x + d along an axis of size n.  Returns -1 if the neighbour lies
   beyond a wall, else the wrapped coordinate. */
static int shift_coord(int x, int d, int n, int wall) {
  int xn = x + d;
  if (xn >= 0 && xn < n) return xn;
  if (wall) return -1;
  return ((xn % n) + n) % n;
}

/* f layout: f[((k * 19 + i) * N) + cell], k = 0 red, 1 blue. */
#define FIDX(k, i, c) ((((long)(k)) * 19 + (i)) * N + (c))

/* Moments of Eq. 4 with the forcing shift: rho_R, rho_B, u. */
static void cell_moments(const or_params *p, const double *f, long N, long c,
                         double *rhoR, double *rhoB, double *u) {
  double rR = 0.0, rB = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 19; ++i) {
    double fr = f[FIDX(0, i, c)], fb = f[FIDX(1, i, c)];
    rR += fr;
    rB += fb;
    for (int a = 0; a < 3; ++a) j[a] += E[i][a] * (fr + fb);
  }
  double rho = rR + rB;
  for (int a = 0; a < 3; ++a) {
    double F = p->force[a] + rho * p->gravity[a];
    u[a] = (j[a] + 0.5 * F) / rho;
  }
  *rhoR = rR;
  *rhoB = rB;
}

int or_moments(const or_params *p, const double *f, double *rho_R,
               double *rho_B, double *u) {
  long N = (long)p->nx * p->ny * p->nz;
  for (long c = 0; c < N; ++c) {
    double uu[3];
    cell_moments(p, f, N, c, &rho_R[c], &rho_B[c], uu);
    for (int a = 0; a < 3; ++a) u[a * N + c] = uu[a];
  }
  return 0;
}

/* Initial populations at equilibrium for given fields (Sec. IV.A: "brought
   to the equilibrium state"). */
int or_init(const or_params *p, const double *rho_R, const double *rho_B,
            const double *u, double *f) {
  long N = (long)p->nx * p->ny * p->nz;
  for (long c = 0; c < N; ++c) {
    double uc[3] = {u[c], u[N + c], u[2 * N + c]};
    double feq[19];
    or_feq(rho_R[c], p->alpha_R, uc, p->improved, p->eq18_coef, feq);
    for (int i = 0; i < 19; ++i) f[FIDX(0, i, c)] = feq[i];
    or_feq(rho_B[c], p->alpha_B, uc, p->improved, p->eq18_coef, feq);
    for (int i = 0; i < 19; ++i) f[FIDX(1, i, c)] = feq[i];
  }
  return 0;
}

/* Eq. 49: d_alpha psi = 3 sum_i omega_i psi(x + e_i) e_{i alpha}, with a
   neighbour beyond a wall replaced by the centre value. */
static double iso_grad(const or_params *p, const double *psi, int x, int y,
                       int z, int axis) {
  double s = 0.0;
  long c0 = cell_index(p, x, y, z);
  for (int i = 1; i < 19; ++i) {
    if (E[i][axis] == 0) continue;
    int xn = shift_coord(x, E[i][0], p->nx, p->wall[0]);
    int yn = shift_coord(y, E[i][1], p->ny, p->wall[1]);
    int zn = shift_coord(z, E[i][2], p->nz, p->wall[2]);
    double v = (xn < 0 || yn < 0 || zn < 0) ? psi[c0]
                                            : psi[cell_index(p, xn, yn, zn)];
    s += weight(i) * v * E[i][axis];
  }
  return 3.0 * s;
}

/* Zou-He velocity nodes on both faces of axis ax (wall = 2): rebuilds, per
   colour, the populations entering from beyond each plate. */
static void zou_he_faces(const or_params *p, double *f, long N, int ax) {
  const int ext[3] = {p->nx, p->ny, p->nz};
  const int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
  for (int side = 0; side < 2; ++side) {
    const int s = side == 0 ? 1 : -1; /* inward normal along ax */
    const double *u = p->wall_u[side];
    const double un = s * u[ax];
    int xyz[3];
    xyz[ax] = side == 0 ? 0 : ext[ax] - 1;
    for (int a = 0; a < ext[t1]; ++a) {
      for (int b = 0; b < ext[t2]; ++b) {
        xyz[t1] = a;
        xyz[t2] = b;
        long c = cell_index(p, xyz[0], xyz[1], xyz[2]);
        for (int k = 0; k < 2; ++k) {
          double s0 = 0.0, sout = 0.0, tang[3] = {0.0, 0.0, 0.0};
          for (int i = 0; i < 19; ++i) {
            const int en = s * E[i][ax];
            const double fi = f[FIDX(k, i, c)];
            if (en == 0) {
              s0 += fi;
              for (int d = 0; d < 3; ++d) tang[d] += E[i][d] * fi;
            } else if (en < 0) {
              sout += fi;
            }
          }
          const double rho = (s0 + 2.0 * sout) / (1.0 - un);
          double Nt[3] = {0.0, 0.0, 0.0};
          Nt[t1] = 0.5 * tang[t1] - rho * u[t1] / 3.0;
          Nt[t2] = 0.5 * tang[t2] - rho * u[t2] / 3.0;
          for (int i = 0; i < 19; ++i) {
            if (s * E[i][ax] != 1) continue;
            double eu = 0.0, corr = 0.0;
            for (int d = 0; d < 3; ++d) {
              eu += E[i][d] * u[d];
              corr += E[i][d] * Nt[d];
            }
            f[FIDX(k, i, c)] = f[FIDX(k, opposite(i), c)] + 6.0 * weight(i) * rho * eu - corr;
          }
        }
      }
    }
  }
}

int or_step(const or_params *p, const double *f_in, double *f_out,
            int nsteps) {
  long N = (long)p->nx * p->ny * p->nz;
  if (N <= 0 || nsteps < 0) return -1;
  double M[361], Minv[361];
  or_matrix_M(M);
  if (or_matrix_Minv(Minv) != 0) return -2;

  double *cur = (double *)malloc(sizeof(double) * 38 * N);
  double *nxt = (double *)malloc(sizeof(double) * 38 * N);
  double *rhoN = (double *)malloc(sizeof(double) * N);
  double *qbar = (double *)malloc(sizeof(double) * 6 * N); /* [k][axis] */
  if (!cur || !nxt || !rhoN || !qbar) {
    free(cur); free(nxt); free(rhoN); free(qbar);
    return -3;
  }
  memcpy(cur, f_in, sizeof(double) * 38 * N);
  const double alpha[2] = {p->alpha_R, p->alpha_B};
  const double Acoef[2] = {p->A_R, p->A_B};

  for (int step = 0; step < nsteps; ++step) {
    /* 1. Moments, rho^N (below Eq. 8) and Qbar^k (below Eq. 49). */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
      double rR, rB, u[3];
      cell_moments(p, cur, N, c, &rR, &rB, u);
      double a = rR / p->rho_in_R, b = rB / p->rho_in_B;
      rhoN[c] = (a - b) / (a + b);
      double rk[2] = {rR, rB};
      for (int k = 0; k < 2; ++k) {
        double cs2 = 0.5 * (1.0 - alpha[k]);
        for (int ax = 0; ax < 3; ++ax)
          qbar[(k * 3 + ax) * N + c] = rk[k] * u[ax] * (1.0 - 3.0 * cs2);
      }
    }

    /* 2. Collision, perturbation, recolouring and streaming per cell. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z) {
      for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
          long c = cell_index(p, x, y, z);
          double rR, rB, u[3];
          cell_moments(p, cur, N, c, &rR, &rB, u);
          double rho = rR + rB;
          double rk[2] = {rR, rB};
          double Ftot[3];
          for (int a = 0; a < 3; ++a)
            Ftot[a] = p->force[a] + rho * p->gravity[a];

          /* Eq. 49: colour gradient and the correction gradients. */
          double grad[3], Q[2][3];
          for (int ax = 0; ax < 3; ++ax) {
            grad[ax] = iso_grad(p, rhoN, x, y, z, ax);
            for (int k = 0; k < 2; ++k)
              Q[k][ax] = iso_grad(p, qbar + (k * 3 + ax) * N, x, y, z, ax);
          }
          if (p->wetting) {
            int side[3] = {0, 0, 0};
            const int xyz[3] = {x, y, z}, ext[3] = {p->nx, p->ny, p->nz};
            for (int a = 0; a < 3; ++a) {
              if (!p->wall[a]) continue;
              if (xyz[a] == 0) side[a] += 1;
              if (xyz[a] == ext[a] - 1) side[a] -= 1;
            }
            or_wetting(side, p->contact_angle_deg, grad);
          }
          double gnorm = sqrt(grad[0] * grad[0] + grad[1] * grad[1] +
                              grad[2] * grad[2]);

          /* Eq. 52 and Eq. 44. */
          double tv = or_tau_v(rhoN[c], p->tau_R, p->tau_B, p->delta);
          double s[19];
          relaxation_diag(p, tv, s);

          double fstar[19];
          for (int i = 0; i < 19; ++i) fstar[i] = 0.0;
          for (int k = 0; k < 2; ++k) {
            double fk[19], mk[19], feq[19], meq[19], Ck[19], Fk[3], Fi[19],
                Fhat[19], mbar[19], om1[19], om2[19], sm[19], om2m[19],
                om2new[19];
            for (int i = 0; i < 19; ++i) fk[i] = cur[FIDX(k, i, c)];
            matvec(M, fk, mk);
            or_feq(rk[k], alpha[k], u, p->improved, p->eq18_coef, feq);
            matvec(M, feq, meq);
            if (p->improved)
              or_correction(Q[k], Ck);
            else
              for (int r = 0; r < 19; ++r) Ck[r] = 0.0;
            for (int a = 0; a < 3; ++a) Fk[a] = (rk[k] / rho) * Ftot[a];
            or_force_guo(Fk, u, Fi);
            matvec(M, Fi, Fhat);
            or_perturbation(Acoef[k], grad, om2); /* Eq. 8 */
            if (p->collision == 1) {
              /* Eq. 20 (BGK), velocity space: relaxation to f^eq at rate
                 1/tau, correction and force under (1 - 1/(2 tau)); the
                 perturbation divided by tau. */
              double Gk[19];
              matvec(Minv, Ck, Gk);
              for (int i = 0; i < 19; ++i) {
                om1[i] = -(fk[i] - feq[i]) / tv + (1.0 - 0.5 / tv) * (Gk[i] + Fi[i]);
                om2new[i] = om2[i] / tv;
              }
            } else {
              /* Eq. 41 (with the forcing term beside the correction). */
              for (int r = 0; r < 19; ++r)
                mbar[r] = -s[r] * (mk[r] - meq[r]) +
                          (1.0 - 0.5 * s[r]) * (Ck[r] + Fhat[r]);
              matvec(Minv, mbar, om1); /* Eq. 42 */
              /* Eq. 53: Lambda = M^-1 S M applied to Omega2. */
              matvec(M, om2, om2m);
              for (int r = 0; r < 19; ++r) sm[r] = s[r] * om2m[r];
              matvec(Minv, sm, om2new);
            }
            /* Eq. 12, summed over colours. */
            for (int i = 0; i < 19; ++i) fstar[i] += fk[i] + om1[i] + om2new[i];
          }

          /* Eq. 10-11: recolouring. */
          for (int i = 0; i < 19; ++i) {
            double cosphi = 0.0;
            if (i > 0 && gnorm >= OR_GRAD_EPS) {
              double eg = E[i][0] * grad[0] + E[i][1] * grad[1] +
                          E[i][2] * grad[2];
              double elen = sqrt((double)(E[i][0] * E[i][0] +
                                          E[i][1] * E[i][1] +
                                          E[i][2] * E[i][2]));
              cosphi = eg / (elen * gnorm);
            }
            double feq0 = rR * phi(i, p->alpha_R) + rB * phi(i, p->alpha_B);
            double seg = p->beta * rR * rB / (rho * rho) * cosphi * feq0;
            double fRp = rR / rho * fstar[i] + seg;
            double fBp = rB / rho * fstar[i] - seg;

            /* Streaming: f^k_i(x + e_i, t + 1) = f^{k,+}_i(x, t), periodic
               wrap or halfway bounce-back at a wall. */
            int xn = shift_coord(x, E[i][0], p->nx, p->wall[0]);
            int yn = shift_coord(y, E[i][1], p->ny, p->wall[1]);
            int zn = shift_coord(z, E[i][2], p->nz, p->wall[2]);
            if (xn < 0 || yn < 0 || zn < 0) {
              int o = opposite(i);
              nxt[FIDX(0, o, c)] = fRp;
              nxt[FIDX(1, o, c)] = fBp;
            } else {
              long cn = cell_index(p, xn, yn, zn);
              nxt[FIDX(0, i, cn)] = fRp;
              nxt[FIDX(1, i, cn)] = fBp;
            }
          }
        }
      }
    }
    /* Moving plates: the populations entering from beyond them. */
    for (int ax = 0; ax < 3; ++ax)
      if (p->wall[ax] == 2) zou_he_faces(p, nxt, N, ax);
    double *t = cur;
    cur = nxt;
    nxt = t;
  }
  memcpy(f_out, cur, sizeof(double) * 38 * N);
  free(cur); free(nxt); free(rhoN); free(qbar);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
