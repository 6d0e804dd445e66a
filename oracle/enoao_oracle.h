/*
 * enoao_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 CPU restatement of the ENO-AO method of H. Shen, "A class
 * of ENO schemes with adaptive order for solving hyperbolic conservation
 * laws" (arXiv 2108.12742).  It exists to check the CUDA library: only the
 * test-suite, the smoke entry and the benchmark's CPU-baseline leg load it.
 * The library never links, includes or calls anything here, and this file
 * shares no header, table or helper with the CUDA path.
 *
 * Layout of a state array: structure of arrays, U[v][k][j][i] with i the
 * fastest index (x), j along y, k along z; v runs over the conserved
 * variables (rho, rho*u, [rho*v], [rho*w], rho*e) for the Euler equations
 * or the single variable u for scalar advection.
 */
#ifndef ENOAO_ORACLE_H
#define ENOAO_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SCALAR = 0, OR_EULER = 1 };
enum { OR_PERIODIC = 0, OR_TRANSMISSIVE = 1 };

typedef struct {
  int ndim;          /* 1, 2 or 3 */
  int system;        /* OR_SCALAR (f = a*u) or OR_EULER */
  int order;         /* designed order, 5 or 7 */
  int nthreads;      /* OpenMP threads for the line loops; <= 0: all */
  long n[3];         /* cells per axis (unused axes: 1) */
  double dx[3];      /* grid spacing per axis */
  int bc[3];         /* OR_PERIODIC or OR_TRANSMISSIVE per axis */
  int alpha_per_stage; /* 0: alpha of U^n for all three stages; 1: each stage
                          takes alpha of its own input state (dt from U^n) */
  int alpha_per_field; /* 0: one alpha per axis for every characteristic field;
                          1 (Euler): field k splits with alpha_k = max over the
                          mesh of |lambda_k| (u_d - c, u_d, ..., u_d + c), the
                          component-wise Lax-Friedrichs reading of Eq.
                          (LF_Flux_Split) applied in characteristic variables */
  double adv_speed;  /* a in f(u) = a*u (scalar only) */
  double gamma;      /* ratio of specific heats (Euler only) */
  double delta;      /* selection threshold of Sec. 3.2 (1e-5 in the paper) */
} or_problem;

/* Number of conserved variables of a problem. */
int or_nvars(const or_problem *P);

/* ENO-AO reconstruction of one interface value f^_{j+1/2} from the window
 * f[k] = f_{j+k}, k = -4..4 (the pointer passed is &f_j; order 5 reads
 * k = -3..3 only).  Writes the chosen candidate's priority index (0..8, see
 * the candidate list in the source), the nine indicators IS (unused ones set
 * to -1) and the smallest relative gap of any comparison that decided the
 * choice (for excusing near-ties).  Returns the reconstructed value. */
double or_face_value(const double *fj, int order, double delta,
                     int *idx, double *is_out, double *gap_rel);

/* Both discrepancies of Eq. (New_Smoothness_Indicator) for candidate c
 * (0..8) on the window f[k] = f_{j+k}; used by the brute-force tests. */
void or_candidate_deltas(const double *fj, int c, double *dl, double *dr);

/* Table-1 value of candidate c on the window f[k] = f_{j+k}. */
double or_candidate_flux(const double *fj, int c);

/* Right / left eigenvector matrices (row-major, nv x nv) of the Euler flux
 * Jacobian along axis 0 at the state (rho, velocity[ndim], H). */
void or_euler_eigen(int ndim, double gamma, const double *vel, double H,
                    double *R, double *L);

/* Roe average (velocity[ndim], H) of two Euler states ql, qr = (rho,
 * momenta..., E) at the face between them (Sec. 4). */
void or_roe_average(const double *ql, const double *qr, int ndim, double gamma,
                    double *vel, double *H);

/* Lax-Friedrichs alpha per axis (max over the mesh of |df/du|). */
int or_alpha(const or_problem *P, const double *U, double *alpha);

/* Per-field splitting constants: alpha_f[d*5 + k] = max over the mesh of
 * |lambda_k| along axis d, with lambda = (u_d - c, u_d, ..., u_d, u_d + c) for
 * the Euler fields (u-c, entropy, shear..., u+c); |a| for scalar advection.
 * Entries beyond ndim / nv are zero. */
int or_alpha_fields(const or_problem *P, const double *U, double *alpha_f);

/* Interface fluxes along axis d for state U with splitting constants alpha.
 * Fhat has the layout of U with n[d] replaced by n[d]+1 faces; face f sits
 * between cells f-1 and f.  idx (nullable) holds, per characteristic field
 * v (u-c, entropy, shear..., u+c; the variable itself for scalars), sign s
 * (0: f^+, 1: f^-) and face, the chosen candidate: idx[(v*2+s)*nf + face]
 * with nf the face count; gap (nullable) holds the decision gap likewise. */
int or_fluxes(const or_problem *P, const double *U, int d, const double *alpha,
              double *Fhat, signed char *idx, double *gap);

/* Spatial operator L(U) of Eq. (1DWENOFD), summed over the axes. */
int or_rhs(const or_problem *P, const double *U, const double *alpha,
           double *rhs);

/* or_fluxes and or_rhs with per-field splitting constants alpha_f (layout of
 * or_alpha_fields): the window's physical fluxes and states are projected
 * separately and field k splits as w^+- = (L_k f +- alpha_k L_k u) / 2. */
int or_fluxes_fields(const or_problem *P, const double *U, int d, const double *alpha_f,
                     double *Fhat, signed char *idx, double *gap);
int or_rhs_fields(const or_problem *P, const double *U, const double *alpha_f,
                  double *rhs);

/* One third-order TVD Runge-Kutta step of size dt, alpha taken from U at the
 * start of the step (and, with alpha_per_stage, from each later stage's
 * input state for that stage); per field with alpha_per_field.  U is updated
 * in place. */
int or_step(const or_problem *P, double *U, double dt);

/* The same step with the splitting constants alpha given for all three
 * stages (alpha is a property of the whole mesh, so a sub-block of a larger
 * grid must be stepped with the full grid's alpha); alpha_per_stage is not
 * consulted. */
int or_step_alpha(const or_problem *P, double *U, double dt, const double *alpha);

/* The same with per-field splitting constants (layout of or_alpha_fields). */
int or_step_alpha_fields(const or_problem *P, double *U, double dt, const double *alpha_f);

/* Advance to t_end.  dt = cfl / sum_d(alpha_d/dx_d) when dt_fixed <= 0,
 * else dt = dt_fixed; the last step is shortened to land on t_end.  Stops
 * early after max_steps steps (max_steps <= 0: no limit). */
int or_advance(const or_problem *P, double *U, double t_end, double cfl,
               double dt_fixed, long max_steps, double *t_out, long *steps_out);

#ifdef __cplusplus
}
#endif
#endif
