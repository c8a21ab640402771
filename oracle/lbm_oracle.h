/*
 * FP64 CPU oracle for the improved 3D colour-gradient MRT lattice Boltzmann
 * step (Wen, Li, Yu, Luo, arXiv:1904.03618).  TEST INFRASTRUCTURE ONLY: used
 * by the tests, the smoke check and the CPU-baseline leg of the benchmark,
 * never by the product path.  Shares nothing with the CUDA sources.
 *
 * Population layout: f[(k * 19 + i) * N + cell], k = 0 red, 1 blue,
 * cell = (z * ny + y) * nx + x.  f holds f_i^k(x, t) after streaming.
 * Field layout: rho[cell], u[axis * N + cell].
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#define OR_GRAD_EPS 1e-12

typedef struct {
  int nx, ny, nz;
  int wall[3];        /* per axis: 0 periodic, 1 halfway bounce-back walls,
                         2 Zou-He velocity nodes (the first and last layer
                         lie on plates moving with wall_u; the other two
                         axes periodic) */
  int improved;       /* 1: Eq. 18 + Eq. 45 correction; 0: Eq. 6, no correction */
  int pad_;
  double rho_in_R, rho_in_B; /* rho_k^in, below Eq. 8 */
  double alpha_R, alpha_B;   /* Eq. 13 */
  double tau_R, tau_B;       /* tau_v^k of Eq. 52 */
  double tau_e, tau_q, tau_pi; /* Eq. 44 */
  double A_R, A_B;           /* Eq. 8 */
  double beta;               /* Eq. 10-11 */
  double delta;              /* Eq. 52 */
  double force[3];           /* uniform force density */
  double gravity[3];         /* acceleration; force density rho * g */
  double eq18_coef;          /* high-order term coefficient of Eq. 18 */
  int wetting;               /* 1: contact-angle rule at wall-adjacent cells */
  int pad2_;
  double contact_angle_deg;  /* theta, measured through the red phase */
  int collision;      /* 0: MRT (Eq. 40-44, 53); 1: BGK with the correction
                         term (Eq. 20) and the perturbation scaled by 1/tau
                         (the treatment above Eq. 53), tau = tau_v of Eq. 52 */
  int pad3_;
  double wall_u[2][3]; /* velocity of the low and high plate of a wall = 2 axis */
} or_params;

void or_matrix_M(double *M);
int or_matrix_Minv(double *Minv);
void or_feq(double rho_k, double alpha_k, const double *u, int improved,
            double eq18_coef, double *feq);
void or_force_guo(const double *Fk, const double *u, double *Fi);
void or_perturbation(double A_k, const double *grad, double *om2);
void or_correction(const double *Q, double *C);
double or_tau_v(double rhoN, double tau_R, double tau_B, double delta);
void or_wetting(const int *wall_side, double theta_deg, double *grad);
int or_moments(const or_params *p, const double *f, double *rho_R,
               double *rho_B, double *u);
int or_init(const or_params *p, const double *rho_R, const double *rho_B,
            const double *u, double *f);
int or_step(const or_params *p, const double *f_in, double *f_out, int nsteps);
int or_num_threads(void);

#endif
