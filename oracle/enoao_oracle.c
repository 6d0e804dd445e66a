/*
 * enoao_oracle.c -- TEST INFRASTRUCTURE ONLY (see enoao_oracle.h).
 *
 * A direct FP64 restatement of Shen's ENO-AO method (arXiv 2108.12742):
 *   Sec. 2    conservative finite-difference form, Eq. (1DWENOFD), global
 *             Lax-Friedrichs splitting, Eq. (LF_Flux_Split), third-order
 *             TVD Runge-Kutta time stepping;
 *   Sec. 3.1  the new smoothness indicator IS = MIN(delta_L, delta_R),
 *             Eq. (New_Smoothness_Indicator), in the closed forms of
 *             Tables 4 and 5;
 *   Sec. 3.2  the candidate sets of ENO-AO5 / ENO-AO7, the interface values
 *             of Table 1 and the selection principle with delta = 1e-5;
 *   Sec. 4    characteristic decomposition with the Roe average at the face.
 * Nothing is blocked, fused or reordered: every interface is computed on its
 * own from its stencil, in the order the paper states the steps.  Compile with
 * -ffp-contract=off so every operation rounds as written.
 */
#include "enoao_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Candidate stencils S_{j-m}^{j+n} of Sec. 3.2 in priority order: a higher   */
/* index has a higher priority (higher order first, and at equal order the     */
/* stencil centred on x_{j+1/2} before the upwind-biased one).  ENO-AO5 uses   */
/* entries 0..5, ENO-AO7 entries 0..8.                                         */
/*   num/den : Table 1, f^_{j+1/2} = sum_i num[i] f_{j-m+i} / den              */
/*   dl      : Table 4, delta_L = |sum_i dl[i] f_{j-m-1+i}|                    */
/*   dr      : Table 5, delta_R = |sum_i dr[i] f_{j-m+i}|                      */
/* S_j^j has its own two-difference form of delta_L / delta_R (Eq.             */
/* New_Smoothness_Indicator, m = n = 0) and no dl/dr entries.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int m, n, den;
  int num[7];
  int dl[8];
  int dr[8];
} cand_t;

static const cand_t CANDS[9] = {
    /* S_j^j        */ {0, 0, 1, {1}, {0}, {0}},
    /* S_j^{j+1}    */ {0, 1, 2, {1, 1}, {1, -2, 1}, {1, -2, 1}},
    /* S_{j-1}^{j+1}*/ {1, 1, 6, {-1, 5, 2}, {-1, 3, -3, 1}, {-1, 3, -3, 1}},
    /* S_{j-2}^{j+1}*/ {2, 1, 12, {1, -5, 13, 3}, {1, -4, 6, -4, 1}, {1, -4, 6, -4, 1}},
    /* S_{j-1}^{j+2}*/ {1, 2, 12, {-1, 7, 7, -1}, {1, -4, 6, -4, 1}, {1, -4, 6, -4, 1}},
    /* S_{j-2}^{j+2}*/ {2, 2, 60, {2, -13, 47, 27, -3},
                        {-1, 5, -10, 10, -5, 1}, {-1, 5, -10, 10, -5, 1}},
    /* S_{j-3}^{j+2}*/ {3, 2, 60, {-1, 7, -23, 57, 22, -2},
                        {1, -6, 15, -20, 15, -6, 1}, {1, -6, 15, -20, 15, -6, 1}},
    /* S_{j-2}^{j+3}*/ {2, 3, 60, {1, -8, 37, 37, -8, 1},
                        {1, -6, 15, -20, 15, -6, 1}, {1, -6, 15, -20, 15, -6, 1}},
    /* S_{j-3}^{j+3}*/ {3, 3, 420, {-3, 25, -101, 319, 214, -38, 4},
                        {-1, 7, -21, 35, -35, 21, -7, 1}, {-1, 7, -21, 35, -35, 21, -7, 1}},
};

static int n_candidates(int order) { return order == 7 ? 9 : 6; }

void or_candidate_deltas(const double *fj, int c, double *dl, double *dr) {
  const cand_t *C = &CANDS[c];
  if (C->m == 0 && C->n == 0) {
    /* two-difference average on each side (Remark after Eq. New_Smoothness_Indicator) */
    *dl = 0.5 * (fabs(fj[0] - fj[-1]) + fabs(fj[-1] - fj[-2]));
    *dr = 0.5 * (fabs(fj[0] - fj[1]) + fabs(fj[1] - fj[2]));
    return;
  }
  int w = C->m + C->n + 2; /* cells in the extended stencil */
  double sl = 0.0, sr = 0.0;
  for (int i = 0; i < w; ++i) sl += C->dl[i] * fj[-C->m - 1 + i];
  for (int i = 0; i < w; ++i) sr += C->dr[i] * fj[-C->m + i];
  *dl = fabs(sl);
  *dr = fabs(sr);
}

double or_candidate_flux(const double *fj, int c) {
  const cand_t *C = &CANDS[c];
  double s = 0.0;
  for (int i = 0; i <= C->m + C->n; ++i) s += C->num[i] * fj[-C->m + i];
  return s / C->den;
}

double or_face_value(const double *fj, int order, double delta, int *idx_out,
                     double *is_out, double *gap_rel) {
  int nc = n_candidates(order);
  double IS[9];
  for (int c = 0; c < 9; ++c) IS[c] = -1.0;
  for (int c = 0; c < nc; ++c) {
    double dl, dr;
    or_candidate_deltas(fj, c, &dl, &dr);
    IS[c] = dl < dr ? dl : dr; /* IS = MIN(delta_L, delta_R) */
  }

  /* Principle 1: among the candidates with IS <= delta the one with the
   * highest priority wins. */
  int pick = -1;
  for (int c = nc - 1; c >= 0; --c)
    if (IS[c] <= delta) { pick = c; break; }
  int threshold_regime = pick >= 0;
  /* Principle 2: otherwise the smallest IS; equal values go to the higher
   * priority (the appendix code scans upward with "<="). */
  if (!threshold_regime) {
    pick = 0;
    for (int c = 1; c < nc; ++c)
      if (IS[c] <= IS[pick]) pick = c;
  }

  if (gap_rel) {
    /* Smallest gap among the comparisons that fixed the choice, relative to
     * the magnitude of the terms that enter an indicator. */
    double fmax = 0.0;
    for (int k = -(order / 2 + 1); k <= order / 2 + 1; ++k)
      if (fabs(fj[k]) > fmax) fmax = fabs(fj[k]);
    double scale = (double)(1 << order) * fmax;
    double gap = INFINITY;
    int lo = threshold_regime ? pick : 0;
    for (int c = lo; c < nc; ++c) {
      double g = fabs(IS[c] - delta);
      if (g < gap) gap = g;
    }
    if (!threshold_regime)
      for (int c = 0; c < nc; ++c)
        if (c != pick) {
          double g = fabs(IS[c] - IS[pick]);
          if (g < gap) gap = g;
        }
    *gap_rel = scale > 0.0 ? gap / scale : INFINITY;
  }
  if (idx_out) *idx_out = pick;
  if (is_out) memcpy(is_out, IS, sizeof IS);
  return or_candidate_flux(fj, pick);
}

/* ------------------------------------------------------------------------ */
/* Physics                                                                   */
/* ------------------------------------------------------------------------ */
int or_nvars(const or_problem *P) { return P->system == OR_EULER ? P->ndim + 2 : 1; }

/* Euler quantities of a state q = (rho, m_normal, m_tangential..., E), i.e.
 * the conserved variables with the momentum along the sweep axis first. */
static double euler_pressure(const double *q, int nv, double gamma) {
  double ke = 0.0;
  for (int i = 1; i < nv - 1; ++i) ke += q[i] * q[i];
  ke = 0.5 * ke / q[0];
  return (gamma - 1.0) * (q[nv - 1] - ke);
}

/* Flux along the sweep axis (Sec. 4.2, F = [rho u, rho u^2 + p, rho u v, (rho e + p) u]). */
static void phys_flux(const or_problem *P, const double *q, int nv, double *F) {
  if (P->system == OR_SCALAR) {
    F[0] = P->adv_speed * q[0];
    return;
  }
  double p = euler_pressure(q, nv, P->gamma);
  double un = q[1] / q[0];
  F[0] = q[1];
  F[1] = q[1] * un + p;
  for (int i = 2; i < nv - 1; ++i) F[i] = q[i] * un;
  F[nv - 1] = (q[nv - 1] + p) * un;
}

void or_euler_eigen(int ndim, double gamma, const double *vel, double H,
                    double *R, double *L) {
  int nv = ndim + 2;
  double q2 = 0.0;
  for (int i = 0; i < ndim; ++i) q2 += vel[i] * vel[i];
  double c2 = (gamma - 1.0) * (H - 0.5 * q2);
  double c = sqrt(c2);
  double u = vel[0];
  double b1 = (gamma - 1.0) / c2;
  double b2 = 0.5 * q2 * b1;
  memset(R, 0, sizeof(double) * nv * nv);
  memset(L, 0, sizeof(double) * nv * nv);
  /* columns of R: 0 = (u - c) wave, 1 = entropy wave, 2.. = shear waves,
   * nv-1 = (u + c) wave */
  int a = 0, e = 1, b = nv - 1;
  R[0 * nv + a] = 1.0;
  R[1 * nv + a] = u - c;
  R[(nv - 1) * nv + a] = H - u * c;
  R[0 * nv + e] = 1.0;
  R[1 * nv + e] = u;
  R[(nv - 1) * nv + e] = 0.5 * q2;
  R[0 * nv + b] = 1.0;
  R[1 * nv + b] = u + c;
  R[(nv - 1) * nv + b] = H + u * c;
  for (int t = 1; t < ndim; ++t) {
    R[(1 + t) * nv + a] = vel[t];
    R[(1 + t) * nv + e] = vel[t];
    R[(1 + t) * nv + b] = vel[t];
    R[(1 + t) * nv + (1 + t)] = 1.0;
    R[(nv - 1) * nv + (1 + t)] = vel[t];
  }
  /* rows of L = R^{-1} */
  L[a * nv + 0] = 0.5 * (b2 + u / c);
  L[a * nv + 1] = 0.5 * (-b1 * u - 1.0 / c);
  L[a * nv + nv - 1] = 0.5 * b1;
  L[e * nv + 0] = 1.0 - b2;
  L[e * nv + 1] = b1 * u;
  L[e * nv + nv - 1] = -b1;
  L[b * nv + 0] = 0.5 * (b2 - u / c);
  L[b * nv + 1] = 0.5 * (-b1 * u + 1.0 / c);
  L[b * nv + nv - 1] = 0.5 * b1;
  for (int t = 1; t < ndim; ++t) {
    L[a * nv + 1 + t] = -0.5 * b1 * vel[t];
    L[e * nv + 1 + t] = b1 * vel[t];
    L[b * nv + 1 + t] = -0.5 * b1 * vel[t];
    L[(1 + t) * nv + 0] = -vel[t];
    L[(1 + t) * nv + 1 + t] = 1.0;
  }
}

/* Roe average of two states (Sec. 4: "the Roe average at the cell face is
 * adopted for characteristic decomposition"). */
static void roe_average(const double *ql, const double *qr, int nv, double gamma,
                        double *vel, double *H) {
  double sl = sqrt(ql[0]), sr = sqrt(qr[0]);
  double pl = euler_pressure(ql, nv, gamma), pr = euler_pressure(qr, nv, gamma);
  double hl = (ql[nv - 1] + pl) / ql[0], hr = (qr[nv - 1] + pr) / qr[0];
  for (int i = 0; i < nv - 2; ++i)
    vel[i] = (sl * (ql[1 + i] / ql[0]) + sr * (qr[1 + i] / qr[0])) / (sl + sr);
  *H = (sl * hl + sr * hr) / (sl + sr);
}

/* Exported form of roe_average for the tests that pin it (the Roe property
 * and the flux Jacobian); ql, qr in conserved order with the momentum along
 * the sweep axis first. */
void or_roe_average(const double *ql, const double *qr, int ndim, double gamma,
                    double *vel, double *H) {
  roe_average(ql, qr, ndim + 2, gamma, vel, H);
}

/* ------------------------------------------------------------------------ */
/* Grid traversal                                                            */
/* ------------------------------------------------------------------------ */
#define GHOST 5 /* widest stencil: f_{j-4} .. f_{j+5} for ENO-AO7 */

static int set_threads(const or_problem *P) {
#ifdef _OPENMP
  return P->nthreads > 0 ? P->nthreads : omp_get_max_threads();
#else
  (void)P;
  return 1;
#endif
}

static long n_cells(const or_problem *P) { return P->n[0] * P->n[1] * P->n[2]; }

/* Linear index of cell (i, j, k). */
static long cell_index(const or_problem *P, long i, long j, long k) {
  return (k * P->n[1] + j) * P->n[0] + i;
}

/* Map a possibly out-of-range index along an axis onto a real cell: periodic
 * wrap or zero-gradient (transmissive) copy. */
static long bc_map(long i, long n, int bc) {
  if (bc == OR_PERIODIC) {
    long r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* Fluxes of one line along axis d.  q holds the line's states with GHOST
 * ghost cells on each side, (n + 2*GHOST) x nv, momentum permuted so that
 * component 1 is the one along d.  Writes (n+1) x nv interface fluxes. */
static void line_fluxes(const or_problem *P, int nv, long n, const double *q,
                        double alpha, const double *alpha_v, double *Fh,
                        signed char *idx_line, double *gap_line, long idx_stride,
                        double *work) {
  const int order = P->order;
  const int reach = order / 2 + 2; /* cells j-reach+1 .. j+reach used by face j+1/2 */
  double *fp = work;               /* split fluxes of the window, [2*reach][nv] */
  double *fm = fp + 2 * reach * nv;
  double *wp = fm + 2 * reach * nv; /* characteristic window, per field */
  double *wm = wp + 16;
  double R[25], L[25], Fk[5];

  for (long f = 0; f <= n; ++f) {
    long j = f - 1; /* face j+1/2 */
    /* split fluxes f^+- = (F +- alpha q)/2 of the window cells; with
     * per-field constants, fp and fm hold F and q themselves and the split
     * follows the projection (alpha differs per field) */
    for (int s = 0; s < 2 * reach; ++s) {
      const double *qk = q + (j - reach + 1 + s + GHOST) * nv;
      phys_flux(P, qk, nv, Fk);
      for (int v = 0; v < nv; ++v) {
        if (alpha_v) {
          fp[s * nv + v] = Fk[v];
          fm[s * nv + v] = qk[v];
        } else {
          fp[s * nv + v] = 0.5 * (Fk[v] + alpha * qk[v]);
          fm[s * nv + v] = 0.5 * (Fk[v] - alpha * qk[v]);
        }
      }
    }
    int euler = P->system == OR_EULER;
    if (euler) {
      double vel[3], H;
      roe_average(q + (j + GHOST) * nv, q + (j + 1 + GHOST) * nv, nv, P->gamma, vel, &H);
      or_euler_eigen(nv - 2, P->gamma, vel, H, R, L);
    }
    double what[5];
    for (int v = 0; v < nv; ++v) {
      /* project the window onto characteristic field v */
      for (int s = 0; s < 2 * reach; ++s) {
        double a = 0.0, b = 0.0;
        if (euler) {
          for (int u = 0; u < nv; ++u) {
            a += L[v * nv + u] * fp[s * nv + u];
            b += L[v * nv + u] * fm[s * nv + u];
          }
        } else {
          a = fp[s * nv + v];
          b = fm[s * nv + v];
        }
        if (alpha_v) { /* a = L_v F, b = L_v q */
          wp[s] = 0.5 * (a + alpha_v[v] * b);
          wm[s] = 0.5 * (a - alpha_v[v] * b);
        } else {
          wp[s] = a;
          wm[s] = b;
        }
      }
      /* f^+ : window centred on cell j, wp[s] is cell j-reach+1+s */
      double win[9], gp, gm;
      int ip, im;
      for (int k = -4; k <= 4; ++k) {
        int s = k + reach - 1;
        win[k + 4] = (s >= 0 && s < 2 * reach) ? wp[s] : 0.0;
      }
      double vp = or_face_value(win + 4, order, P->delta, &ip, NULL, &gp);
      /* f^- : the mirror image about x_{j+1/2}, centred on cell j+1 */
      for (int k = -4; k <= 4; ++k) {
        int s = (1 - k) + reach - 1;
        win[k + 4] = (s >= 0 && s < 2 * reach) ? wm[s] : 0.0;
      }
      double vm = or_face_value(win + 4, order, P->delta, &im, NULL, &gm);
      what[v] = vp + vm;
      if (idx_line) {
        idx_line[(v * 2 + 0) * idx_stride + f] = (signed char)ip;
        idx_line[(v * 2 + 1) * idx_stride + f] = (signed char)im;
      }
      if (gap_line) {
        gap_line[(v * 2 + 0) * idx_stride + f] = gp;
        gap_line[(v * 2 + 1) * idx_stride + f] = gm;
      }
    }
    /* back to physical space */
    for (int u = 0; u < nv; ++u) {
      if (euler) {
        double a = 0.0;
        for (int v = 0; v < nv; ++v) a += R[u * nv + v] * what[v];
        Fh[f * nv + u] = a;
      } else {
        Fh[f * nv + u] = what[u];
      }
    }
  }
}

/* Conserved-variable component stored at position c of the permuted line
 * state for a sweep along axis d (momentum along d comes first). */
static int perm_component(int system, int ndim, int d, int c) {
  if (system != OR_EULER || c == 0 || c == ndim + 1) return c;
  int m = c - 1; /* 0 = normal, 1.. = tangential in cyclic order */
  return 1 + (d + m) % ndim;
}

typedef struct {
  const or_problem *P;
  int d, nv;
  long n;       /* cells along d */
  long nlines;  /* lines along d */
} sweep_t;

/* Cell (i,j,k) of the s-th cell of line l along axis d. */
static long line_cell(const or_problem *P, int d, long l, long s) {
  long i, j, k;
  if (d == 0) {
    i = s; j = l % P->n[1]; k = l / P->n[1];
  } else if (d == 1) {
    i = l % P->n[0]; j = s; k = l / P->n[0];
  } else {
    i = l % P->n[0]; j = l / P->n[0]; k = s;
  }
  return cell_index(P, i, j, k);
}

/* Face-array index of face f of line l along axis d (faces replace cells
 * along d, n[d]+1 of them). */
static long line_face(const or_problem *P, int d, long l, long f) {
  long nf0 = P->n[0] + (d == 0), nf1 = P->n[1] + (d == 1);
  long i, j, k;
  if (d == 0) {
    i = f; j = l % P->n[1]; k = l / P->n[1];
  } else if (d == 1) {
    i = l % P->n[0]; j = f; k = l / P->n[0];
  } else {
    i = l % P->n[0]; j = l / P->n[0]; k = f;
  }
  return (k * nf1 + j) * nf0 + i;
}

static void load_line(const or_problem *P, const double *U, int d, long l,
                      int nv, double *q) {
  long n = P->n[d], N = n_cells(P);
  for (long s = -GHOST; s < n + GHOST; ++s) {
    long cell = line_cell(P, d, l, bc_map(s, n, P->bc[d]));
    for (int c = 0; c < nv; ++c)
      q[(s + GHOST) * nv + c] = U[perm_component(P->system, P->ndim, d, c) * N + cell];
  }
}

/* alpha: one constant per axis, or (alpha_f non-null) per axis and field */
static int fluxes_impl(const or_problem *P, const double *U, int d, const double *alpha,
                       const double *alpha_f, double *Fhat, signed char *idx, double *gap) {
  if (d < 0 || d >= P->ndim) return 1;
  int nv = or_nvars(P);
  long n = P->n[d], nlines = n_cells(P) / n;
  long nfaces = nlines * (n + 1);
  int nt = set_threads(P);
#pragma omp parallel num_threads(nt)
  {
    double *q = malloc(sizeof(double) * (n + 2 * GHOST) * nv);
    double *Fh = malloc(sizeof(double) * (n + 1) * nv);
    signed char *il = idx ? malloc((size_t)nv * 2 * (n + 1)) : NULL;
    double *gl = gap ? malloc(sizeof(double) * nv * 2 * (n + 1)) : NULL;
    double work[4 * 10 * 5 + 32];
#pragma omp for schedule(static)
    for (long l = 0; l < nlines; ++l) {
      load_line(P, U, d, l, nv, q);
      line_fluxes(P, nv, n, q, alpha_f ? 0.0 : alpha[d], alpha_f ? alpha_f + 5 * d : NULL, Fh,
                  il, gl, n + 1, work);
      for (long f = 0; f <= n; ++f) {
        long fi = line_face(P, d, l, f);
        for (int c = 0; c < nv; ++c) {
          int comp = perm_component(P->system, P->ndim, d, c);
          Fhat[comp * nfaces + fi] = Fh[f * nv + c];
        }
        /* choices are stored per characteristic field, in the order
         * (u-c, entropy, shear..., u+c) for the Euler equations */
        for (int c = 0; c < nv && (il || gl); ++c)
          for (int s = 0; s < 2; ++s) {
            if (il) idx[(c * 2 + s) * nfaces + fi] = il[(c * 2 + s) * (n + 1) + f];
            if (gl) gap[(c * 2 + s) * nfaces + fi] = gl[(c * 2 + s) * (n + 1) + f];
          }
      }
    }
    free(q);
    free(Fh);
    free(il);
    free(gl);
  }
  return 0;
}

int or_fluxes(const or_problem *P, const double *U, int d, const double *alpha,
              double *Fhat, signed char *idx, double *gap) {
  return fluxes_impl(P, U, d, alpha, NULL, Fhat, idx, gap);
}

int or_fluxes_fields(const or_problem *P, const double *U, int d, const double *alpha_f,
                     double *Fhat, signed char *idx, double *gap) {
  return fluxes_impl(P, U, d, NULL, alpha_f, Fhat, idx, gap);
}

static int rhs_impl(const or_problem *P, const double *U, const double *alpha,
                    const double *alpha_f, double *rhs) {
  int nv = or_nvars(P);
  long N = n_cells(P);
  memset(rhs, 0, sizeof(double) * nv * N);
  for (int d = 0; d < P->ndim; ++d) {
    long n = P->n[d], nlines = N / n;
    double dx = P->dx[d];
    int nt = set_threads(P);
#pragma omp parallel num_threads(nt)
    {
      double *q = malloc(sizeof(double) * (n + 2 * GHOST) * nv);
      double *Fh = malloc(sizeof(double) * (n + 1) * nv);
      double work[4 * 10 * 5 + 32];
#pragma omp for schedule(static)
      for (long l = 0; l < nlines; ++l) {
        load_line(P, U, d, l, nv, q);
        line_fluxes(P, nv, n, q, alpha_f ? 0.0 : alpha[d], alpha_f ? alpha_f + 5 * d : NULL, Fh,
                    NULL, NULL, n + 1, work);
        for (long s = 0; s < n; ++s) {
          long cell = line_cell(P, d, l, s);
          for (int c = 0; c < nv; ++c) {
            int comp = perm_component(P->system, P->ndim, d, c);
            /* L(u)_j = -(f^_{j+1/2} - f^_{j-1/2}) / dx, Eq. (1DWENOFD) */
            rhs[comp * N + cell] += -(Fh[(s + 1) * nv + c] - Fh[s * nv + c]) / dx;
          }
        }
      }
      free(q);
      free(Fh);
    }
  }
  return 0;
}

int or_rhs(const or_problem *P, const double *U, const double *alpha, double *rhs) {
  return rhs_impl(P, U, alpha, NULL, rhs);
}

int or_rhs_fields(const or_problem *P, const double *U, const double *alpha_f, double *rhs) {
  return rhs_impl(P, U, NULL, alpha_f, rhs);
}

int or_alpha_fields(const or_problem *P, const double *U, double *alpha_f) {
  long N = n_cells(P);
  int nv = or_nvars(P);
  for (int i = 0; i < 15; ++i) alpha_f[i] = 0.0;
  if (P->system == OR_SCALAR) {
    for (int d = 0; d < P->ndim; ++d) alpha_f[5 * d] = fabs(P->adv_speed);
    return 0;
  }
  for (long c = 0; c < N; ++c) {
    double q[5];
    for (int v = 0; v < nv; ++v) q[v] = U[v * N + c];
    double p = euler_pressure(q, nv, P->gamma);
    if (!(q[0] > 0.0) || !(p > 0.0)) return 2; /* non-physical state */
    double a = sqrt(P->gamma * p / q[0]);
    for (int d = 0; d < P->ndim; ++d) {
      double u = q[1 + d] / q[0];
      /* eigenvalues of the flux Jacobian along d, fields (u-c, entropy, shear..., u+c) */
      for (int k = 0; k < nv; ++k) {
        double lam = k == 0 ? u - a : (k == nv - 1 ? u + a : u);
        if (fabs(lam) > alpha_f[5 * d + k]) alpha_f[5 * d + k] = fabs(lam);
      }
    }
  }
  return 0;
}

int or_alpha(const or_problem *P, const double *U, double *alpha) {
  long N = n_cells(P);
  int nv = or_nvars(P);
  for (int d = 0; d < 3; ++d) alpha[d] = 0.0;
  if (P->system == OR_SCALAR) {
    for (int d = 0; d < P->ndim; ++d) alpha[d] = fabs(P->adv_speed);
    return 0;
  }
  for (long c = 0; c < N; ++c) {
    double q[5];
    for (int v = 0; v < nv; ++v) q[v] = U[v * N + c];
    double p = euler_pressure(q, nv, P->gamma);
    if (!(q[0] > 0.0) || !(p > 0.0)) return 2; /* non-physical state */
    double a = sqrt(P->gamma * p / q[0]);
    for (int d = 0; d < P->ndim; ++d) {
      double s = fabs(q[1 + d] / q[0]) + a;
      if (s > alpha[d]) alpha[d] = s;
    }
  }
  return 0;
}

/* The three stages of the third-order TVD Runge-Kutta scheme (Sec. 2).
 * Stage 0 splits with alpha0 (3 values, or 15 per field with per_field);
 * with per_stage set, stages 1 and 2 split with the alpha of their own input
 * state (u1, u2) instead. */
static int rk3_step(const or_problem *P, double *U, double dt, const double *alpha0,
                    int per_stage, int per_field) {
  int nv = or_nvars(P);
  long M = (long)nv * n_cells(P);
  double *u0 = malloc(sizeof(double) * M);
  double *L = malloc(sizeof(double) * M);
  double alpha[15];
  for (int i = 0; i < (per_field ? 15 : 3); ++i) alpha[i] = alpha0[i];
  int st = 0;
#define OR_STAGE_ALPHA() (per_field ? or_alpha_fields(P, U, alpha) : or_alpha(P, U, alpha))
#define OR_STAGE_RHS() (per_field ? or_rhs_fields(P, U, alpha, L) : or_rhs(P, U, alpha, L))
  memcpy(u0, U, sizeof(double) * M);
  /* u1 = u0 + dt L(u0) */
  OR_STAGE_RHS();
  for (long i = 0; i < M; ++i) U[i] = u0[i] + dt * L[i];
  /* u2 = 3/4 u0 + 1/4 (u1 + dt L(u1)) */
  if (per_stage) st = OR_STAGE_ALPHA();
  if (!st) {
    OR_STAGE_RHS();
    for (long i = 0; i < M; ++i) U[i] = 0.75 * u0[i] + 0.25 * (U[i] + dt * L[i]);
    /* u^{n+1} = 1/3 u0 + 2/3 (u2 + dt L(u2)) */
    if (per_stage) st = OR_STAGE_ALPHA();
  }
  if (!st) {
    OR_STAGE_RHS();
    for (long i = 0; i < M; ++i)
      U[i] = (1.0 / 3.0) * u0[i] + (2.0 / 3.0) * (U[i] + dt * L[i]);
  }
#undef OR_STAGE_ALPHA
#undef OR_STAGE_RHS
  free(u0);
  free(L);
  return st;
}

int or_step(const or_problem *P, double *U, double dt) {
  const int euler = P->system == OR_EULER;
  double alpha[15];
  int st = P->alpha_per_field && euler ? or_alpha_fields(P, U, alpha) : or_alpha(P, U, alpha);
  if (st) return st;
  return rk3_step(P, U, dt, alpha, P->alpha_per_stage && euler, P->alpha_per_field && euler);
}

int or_step_alpha(const or_problem *P, double *U, double dt, const double *alpha) {
  return rk3_step(P, U, dt, alpha, 0, 0);
}

int or_step_alpha_fields(const or_problem *P, double *U, double dt, const double *alpha_f) {
  return rk3_step(P, U, dt, alpha_f, 0, 1);
}

int or_advance(const or_problem *P, double *U, double t_end, double cfl,
               double dt_fixed, long max_steps, double *t_out, long *steps_out) {
  double t = 0.0;
  long steps = 0;
  int st = 0;
  while (t < t_end && (max_steps <= 0 || steps < max_steps)) {
    double dt;
    if (dt_fixed > 0.0) {
      dt = dt_fixed;
    } else {
      double alpha[3], s = 0.0;
      st = or_alpha(P, U, alpha);
      if (st) break;
      for (int d = 0; d < P->ndim; ++d) s += alpha[d] / P->dx[d];
      dt = cfl / s;
    }
    int last = 0;
    if (t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    st = or_step(P, U, dt);
    if (st) break;
    t = last ? t_end : t + dt;
    ++steps;
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  return st;
}
