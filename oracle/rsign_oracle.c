/*
 * rsign_oracle.c -- plain, slow, FP64 CPU oracle for the shifted matrix-sign
 * reflector R_k = I - 2 P_k = sign(H - s I).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call into this file.  It shares no code,
 * header, table or helper with the CUDA library; it is compiled on its own
 * with plain gcc (OpenMP optional).
 *
 * Contents, each written out from the definition it cites:
 *   - cyclic Jacobi eigen-decomposition of a symmetric matrix (the spectral
 *     decomposition H = Q Lambda Q^T with ascending eigenvalues, Sec. 2.1);
 *   - the reflector R_k = I - 2 Q_k Q_k^T from an eigenbasis (Eq. Pk and
 *     Eq. Rk_intro; Prop. 2.1 makes it equal to sign(H - sI));
 *   - the Gershgorin / infinity-norm scaling alpha = 1/||A||_inf (Sec. 4.3,
 *     "cheaper surrogate" of 1/||H - sI||_2);
 *   - a naive FP64 Newton-Schulz loop X_{m+1} = 1/2 X_m (3I - X_m^2),
 *     X_0 = alpha A (Eq. NS), row by row;
 *   - the Daleckii-Krein form of the Frechet derivative of sign(A) along a
 *     symmetric direction W: Q (F o Q^T W Q) Q^T with
 *     F_ij = (sign mu_i - sign mu_j)/(mu_i - mu_j), used to check gradients.
 *
 * Conventions: matrices are dense row-major d x d, leading dimension d.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int rsign_oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Cyclic Jacobi (Sec. 2.1: H = Q diag(lambda) Q^T, lambda ascending).      */
/* ---------------------------------------------------------------------- */

static double off_norm2(int64_t d, const double *A) {
  double s = 0.0;
  for (int64_t i = 0; i < d; ++i)
    for (int64_t j = 0; j < d; ++j)
      if (i != j) s += A[i * d + j] * A[i * d + j];
  return s;
}

/*
 * Eigen-decomposition of the symmetric part of A_in by row-cyclic Jacobi
 * sweeps.  Each rotation in the (p, q) plane is chosen to annihilate a_pq:
 * with theta = (a_qq - a_pp) / (2 a_pq) the tangent of the rotation angle is
 * t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(1 + t^2),
 * s = t c.  The full matrix is updated (rows and columns p, q), and the
 * rotations are accumulated into V.  Sweeps stop when
 * off(A) <= tol * ||A||_F or after max_sweeps.
 *
 * Output: lam[0..d-1] ascending (ties broken by original index), and V with
 * column i (V[r*d + i]) the unit eigenvector of lam[i].
 * Returns the number of sweeps used, or -1 if not converged.
 */
int rsign_oracle_jacobi(int64_t d, const double *A_in, double *lam, double *V,
                        int max_sweeps, double tol) {
  double *A = (double *)malloc(sizeof(double) * d * d);
  double *W = (double *)malloc(sizeof(double) * d * d);
  if (!A || !W) { free(A); free(W); return -2; }
  for (int64_t i = 0; i < d; ++i)
    for (int64_t j = 0; j < d; ++j)
      A[i * d + j] = 0.5 * (A_in[i * d + j] + A_in[j * d + i]);
  for (int64_t i = 0; i < d * d; ++i) W[i] = 0.0;
  for (int64_t i = 0; i < d; ++i) W[i * d + i] = 1.0;

  double fro2 = 0.0;
  for (int64_t i = 0; i < d * d; ++i) fro2 += A[i] * A[i];
  const double target = tol * tol * fro2;

  int sweeps = 0, converged = 0;
  for (; sweeps < max_sweeps; ++sweeps) {
    if (off_norm2(d, A) <= target) { converged = 1; break; }
    for (int64_t p = 0; p < d - 1; ++p) {
      for (int64_t q = p + 1; q < d; ++q) {
        const double apq = A[p * d + q];
        if (apq == 0.0) continue;
        const double app = A[p * d + p], aqq = A[q * d + q];
        const double theta = (aqq - app) / (2.0 * apq);
        double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
        if (theta < 0.0) t = -t;
        const double c = 1.0 / sqrt(t * t + 1.0);
        const double s = t * c;
        /* rotate columns p and q: A <- A J */
        for (int64_t r = 0; r < d; ++r) {
          const double arp = A[r * d + p], arq = A[r * d + q];
          A[r * d + p] = c * arp - s * arq;
          A[r * d + q] = s * arp + c * arq;
        }
        /* rotate rows p and q: A <- J^T A */
        for (int64_t r = 0; r < d; ++r) {
          const double apr = A[p * d + r], aqr = A[q * d + r];
          A[p * d + r] = c * apr - s * aqr;
          A[q * d + r] = s * apr + c * aqr;
        }
        A[p * d + q] = 0.0;
        A[q * d + p] = 0.0;
        /* accumulate: W <- W J */
        for (int64_t r = 0; r < d; ++r) {
          const double wrp = W[r * d + p], wrq = W[r * d + q];
          W[r * d + p] = c * wrp - s * wrq;
          W[r * d + q] = s * wrp + c * wrq;
        }
      }
    }
  }
  if (!converged && off_norm2(d, A) <= target) converged = 1;

  /* sort ascending by eigenvalue, stable in the original index */
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * d);
  for (int64_t i = 0; i < d; ++i) ord[i] = i;
  for (int64_t i = 1; i < d; ++i) { /* insertion sort: plain and stable */
    int64_t key = ord[i];
    int64_t j = i - 1;
    while (j >= 0 && A[ord[j] * d + ord[j]] > A[key * d + key]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = key;
  }
  for (int64_t i = 0; i < d; ++i) {
    lam[i] = A[ord[i] * d + ord[i]];
    for (int64_t r = 0; r < d; ++r) V[r * d + i] = W[r * d + ord[i]];
  }
  free(ord);
  free(A);
  free(W);
  return converged ? sweeps : -1;
}

/* ---------------------------------------------------------------------- */
/* Reflector from an eigenbasis: R_k = I - 2 Q_k Q_k^T (Eq. Pk, Rk_intro).  */
/* ---------------------------------------------------------------------- */
void rsign_oracle_reflector_from_basis(int64_t d, int64_t k, const double *V, double *R) {
  for (int64_t i = 0; i < d; ++i) {
    for (int64_t j = 0; j < d; ++j) {
      double p = 0.0;
      for (int64_t l = 0; l < k; ++l) p += V[i * d + l] * V[j * d + l];
      R[i * d + j] = (i == j ? 1.0 : 0.0) - 2.0 * p;
    }
  }
  /* the definition is symmetric; make the stored copy symmetric bitwise */
  for (int64_t i = 0; i < d; ++i)
    for (int64_t j = i + 1; j < d; ++j) {
      const double a = 0.5 * (R[i * d + j] + R[j * d + i]);
      R[i * d + j] = a;
      R[j * d + i] = a;
    }
}

/* ---------------------------------------------------------------------- */
/* Scaling alpha = 1 / ||A||_inf  (Sec. 4.3 discussion of scaling choices).  */
/* For symmetric A this is the Gershgorin bound on rho(A).                   */
/* ---------------------------------------------------------------------- */
double rsign_oracle_inf_norm(int64_t d, const double *A) {
  double m = 0.0;
  for (int64_t i = 0; i < d; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < d; ++j) s += fabs(A[i * d + j]);
    if (s > m) m = s;
  }
  return m;
}

/* ---------------------------------------------------------------------- */
/* Naive Newton-Schulz, Eq. NS:  X_{m+1} = 1/2 X_m (3 I - X_m^2).           */
/* ---------------------------------------------------------------------- */

/*
 * One Newton-Schulz step restricted to rows [row0, row1):
 *   Z_i = X_i X        (row i of X^2)
 *   Xn_i = 1/2 (3 X_i - Z_i X)
 * and the contribution of those rows to ||X^2 - I||_F^2 is returned.
 * Row i of the product needs only row i of X and the whole of X, so rows are
 * independent (OpenMP over rows).
 */
double rsign_oracle_ns_step_rows(int64_t d, const double *X, double *Xn, int64_t row0, int64_t row1) {
  double res2 = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : res2)
  for (int64_t i = row0; i < row1; ++i) {
    double *Z = (double *)calloc((size_t)d, sizeof(double));
    double *T = (double *)calloc((size_t)d, sizeof(double));
    for (int64_t k = 0; k < d; ++k) {
      const double a = X[i * d + k];
      for (int64_t j = 0; j < d; ++j) Z[j] += a * X[k * d + j];
    }
    for (int64_t j = 0; j < d; ++j) {
      const double e = Z[j] - (i == j ? 1.0 : 0.0);
      res2 += e * e;
    }
    for (int64_t k = 0; k < d; ++k) {
      const double a = Z[k];
      for (int64_t j = 0; j < d; ++j) T[j] += a * X[k * d + j];
    }
    for (int64_t j = 0; j < d; ++j) Xn[i * d + j] = 0.5 * (3.0 * X[i * d + j] - T[j]);
    free(Z);
    free(T);
  }
  return res2;
}

/*
 * Newton-Schulz from X0 (already scaled: X0 = alpha (H - sI)).
 * At step m the residual r_m = ||X_m^2 - I||_F is formed; if r_m < tol the
 * loop stops and X = X_m is returned, otherwise X_{m+1} is formed.  At most
 * max_steps updates are applied.  resid_hist[m] receives r_m (length
 * max_steps + 1, may be NULL).  Returns the number of updates applied (m);
 * *converged is set to 1 if the tolerance was met.
 */
int rsign_oracle_newton_schulz(int64_t d, const double *X0, double *X, double tol, int max_steps,
                               double *resid_hist, int *converged) {
  double *Xc = (double *)malloc(sizeof(double) * d * d);
  double *Xn = (double *)malloc(sizeof(double) * d * d);
  memcpy(Xc, X0, sizeof(double) * d * d);
  int m = 0;
  *converged = 0;
  for (;; ++m) {
    const double r = sqrt(rsign_oracle_ns_step_rows(d, Xc, Xn, 0, d));
    if (resid_hist) resid_hist[m] = r;
    if (r < tol) { *converged = 1; break; }
    if (m == max_steps) break;
    double *t = Xc; Xc = Xn; Xn = t;
  }
  memcpy(X, Xc, sizeof(double) * d * d);
  free(Xc);
  free(Xn);
  return m;
}

/* ---------------------------------------------------------------------- */
/* Dense products used by the checks (plain triple loops).                  */
/* ---------------------------------------------------------------------- */
void rsign_oracle_matmul(int64_t n, int64_t kdim, int64_t m, const double *A, const double *B, double *C) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < m; ++j) C[i * m + j] = 0.0;
    for (int64_t k = 0; k < kdim; ++k) {
      const double a = A[i * kdim + k];
      for (int64_t j = 0; j < m; ++j) C[i * m + j] += a * B[k * m + j];
    }
  }
}

/* ---------------------------------------------------------------------- */
/* Daleckii-Krein: derivative of sign(A) along symmetric W, for the         */
/* eigen-decomposition A = V diag(mu) V^T:                                  */
/*   L(A, W) = V (F o (V^T W V)) V^T,                                       */
/*   F_ij = (sign mu_i - sign mu_j) / (mu_i - mu_j), 0 when the signs agree. */
/* With W the adjoint seed Gbar, <Gbar, L(A, dA)> = <L(A, Gbar), dA>, so the */
/* same routine gives the gradient of <Gbar, sign(A)> with respect to A.    */
/* ---------------------------------------------------------------------- */
void rsign_oracle_daleckii_krein(int64_t d, const double *mu, const double *V, const double *W, double *out) {
  double *T = (double *)malloc(sizeof(double) * d * d);
  double *M = (double *)malloc(sizeof(double) * d * d);
  double *Vt = (double *)malloc(sizeof(double) * d * d);
  for (int64_t i = 0; i < d; ++i)
    for (int64_t j = 0; j < d; ++j) Vt[i * d + j] = V[j * d + i];
  rsign_oracle_matmul(d, d, d, Vt, W, T); /* V^T W */
  rsign_oracle_matmul(d, d, d, T, V, M);  /* V^T W V */
  for (int64_t i = 0; i < d; ++i)
    for (int64_t j = 0; j < d; ++j) {
      const double si = mu[i] > 0 ? 1.0 : -1.0, sj = mu[j] > 0 ? 1.0 : -1.0;
      const double f = (si == sj) ? 0.0 : (si - sj) / (mu[i] - mu[j]);
      M[i * d + j] *= f;
    }
  rsign_oracle_matmul(d, d, d, V, M, T);  /* V (F o ...) */
  rsign_oracle_matmul(d, d, d, T, Vt, out);
  free(T);
  free(M);
  free(Vt);
}
