/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU oracle for dense Tucker
 * decomposition by STHOSVD + HOOI.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this file.  It
 * shares no code, header, table or helper with the CUDA path and never calls
 * into it.
 *
 * Conventions (the paper leaves the unfolding column order open, Sec. 2.1
 * "Tensor Unfolding"; the result does not depend on it):
 *   - a tensor of size L_0 x ... x L_{N-1} is stored row-major (C order),
 *     mode N-1 fastest; modes are numbered from 0 here (the paper counts 1..N);
 *   - a factor matrix F_n (L_n x K_n, Sec. 2.2) is row-major;
 *   - all arithmetic is in double.  The input tensor may be given as float
 *     (the values a GPU sees) or double.
 *
 * Functions and the passage each follows:
 *   orc_ttm_*        Sec. 2.1 "Tensor-Times-Matrix": Z = X x_n A, A of size
 *                    Kout x L_n, applied to every mode-n fiber (literal sum).
 *   orc_gram         Sec. 5 (SVD via Gram matrix A A^T then EVD): W = Z_(n) Z_(n)^T.
 *   orc_jacobi_eig   the EVD of Sec. 5, here by the classical cyclic Jacobi
 *                    method (the paper calls LAPACK's dsyevx; any exact
 *                    symmetric eigensolver gives the same eigenpairs).
 *   orc_hooi_sweep   Fig. 2 "HOOI Procedure": for each n, Z <- T x_{j!=n} F_j^T
 *                    with the INPUT factors, F~_n <- leading K_n left singular
 *                    vectors of Z_(n); then G~ <- T x_1 F~_1^T ... x_N F~_N^T.
 *                    Chains run in natural mode order (chain trees, Sec. 3.2).
 *                    A Gauss-Seidel variant (updated factors for j < n) is
 *                    kept as a cross-check only.
 *   orc_sthosvd      STHOSVD (Sec. 1/2.2 cite it; standard definition):
 *                    natural mode order, Gram + EVD per mode, then truncate.
 *   orc_sthosvd_order  the same with the modes in a given order (the
 *                    STHOSVD order optimisation, to which Sec. 1 says the
 *                    tree ideas carry over, picks one).
 *   orc_core         Fig. 2 "New core".
 *   orc_fit          Sec. 2.2 error "normalized root mean square":
 *                    rel = ||T - Z||_F / ||T||_F, fit = 1 - rel, using
 *                    ||T - G x F||^2 = ||T||^2 - ||G||^2 for orthonormal F.
 *   orc_residual     the same error by direct reconstruction (small sizes).
 *
 * Eigenvector convention (the paper fixes none): eigenpairs sorted by
 * descending eigenvalue; each eigenvector's entry of largest magnitude
 * (lowest row on ties) is made positive.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* L_0 + ... + L_{n-1} */
static int64_t len_sum(const int64_t* d, int n) {
  int64_t s = 0;
  for (int i = 0; i < n; ++i) s += d[i];
  return s;
}

static int64_t prod_range(const int64_t* d, int a, int b) {
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= d[i];
  return p;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * TTM (Sec. 2.1): Y = X x_n A with A of size Kout x L_n (row-major).
 * Y[r, k, c] = sum_l A[k, l] * X[r, l, c], where r runs over the modes before
 * n and c over the modes after n.
 * ------------------------------------------------------------------------- */
#define ORC_TTM_BODY(XT)                                                        \
  const int64_t R = prod_range(dims, 0, n);                                     \
  const int64_t Ln = dims[n];                                                   \
  const int64_t C = prod_range(dims, n + 1, N);                                 \
  _Pragma("omp parallel for collapse(2) schedule(static)")                      \
  for (int64_t r = 0; r < R; ++r) {                                             \
    for (int64_t k = 0; k < Kout; ++k) {                                        \
      double* y = Y + (r * Kout + k) * C;                                       \
      for (int64_t c = 0; c < C; ++c) y[c] = 0.0;                               \
      for (int64_t l = 0; l < Ln; ++l) {                                        \
        const double a = A[k * Ln + l];                                         \
        const XT* x = X + (r * Ln + l) * C;                                     \
        for (int64_t c = 0; c < C; ++c) y[c] += a * (double)x[c];              \
      }                                                                         \
    }                                                                           \
  }

void orc_ttm_d(int N, const int64_t* dims, const double* X, int n,
               const double* A, int64_t Kout, double* Y) {
  ORC_TTM_BODY(double)
}

void orc_ttm_f(int N, const int64_t* dims, const float* X, int n,
               const double* A, int64_t Kout, double* Y) {
  ORC_TTM_BODY(float)
}

/* Fig. 2 uses T x_j F_j^T: transpose the L_j x K_j factor into K_j x L_j. */
static double* transpose_factor(const double* F, int64_t L, int64_t K) {
  double* Ft = (double*)malloc(sizeof(double) * (size_t)(L * K));
  for (int64_t l = 0; l < L; ++l)
    for (int64_t k = 0; k < K; ++k) Ft[k * L + l] = F[l * K + k];
  return Ft;
}

/* Gram of the mode-n unfolding (Sec. 5): W[a, b] = sum over all fibers of
 * Z[.., a, ..] * Z[.., b, ..]. */
void orc_gram(int N, const int64_t* dims, const double* Z, int n, double* W) {
  const int64_t R = prod_range(dims, 0, n);
  const int64_t Ln = dims[n];
  const int64_t C = prod_range(dims, n + 1, N);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t a = 0; a < Ln; ++a) {
    for (int64_t b = 0; b < Ln; ++b) {
      double s = 0.0;
      for (int64_t r = 0; r < R; ++r) {
        const double* za = Z + (r * Ln + a) * C;
        const double* zb = Z + (r * Ln + b) * C;
        for (int64_t c = 0; c < C; ++c) s += za[c] * zb[c];
      }
      W[a * Ln + b] = s;
    }
  }
}

/* ---------------------------------------------------------------------------
 * Cyclic Jacobi eigenvalue method for a real symmetric matrix (row-cyclic
 * ordering; rotation angle chosen as the smaller root so that the (p,q)
 * entry is annihilated).  A (n x n, row-major) is not modified.
 * evals[j] descending; V (n x n row-major) holds eigenvector j in column j.
 * Returns the number of sweeps used, or -1 if it did not converge.
 * ------------------------------------------------------------------------- */
int orc_jacobi_eig(int64_t n, const double* Ain, double* evals, double* V) {
  double* A = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* Q = (double*)malloc(sizeof(double) * (size_t)(n * n));
  memcpy(A, Ain, sizeof(double) * (size_t)(n * n));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) Q[i * n + j] = (i == j) ? 1.0 : 0.0;

  int sweeps = 0, converged = 0;
  for (sweeps = 1; sweeps <= 100; ++sweeps) {
    int rotated = 0;
    for (int64_t p = 0; p < n - 1; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        const double app = A[p * n + p], aqq = A[q * n + q];
        /* relative threshold: skip entries already negligible against the
         * diagonal (Demmel-Veselic criterion) */
        if (apq == 0.0) continue;
        if (fabs(apq) <= 1e-17 * sqrt(fabs(app) * fabs(aqq))) {
          A[p * n + q] = A[q * n + p] = 0.0;
          continue;
        }
        rotated = 1;
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                      : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = t * c;
        /* A <- A J (columns p, q) */
        for (int64_t k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        /* A <- J^T A (rows p, q) */
        for (int64_t k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        A[p * n + q] = A[q * n + p] = 0.0;
        /* Q <- Q J */
        for (int64_t k = 0; k < n; ++k) {
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
    }
    if (!rotated) { converged = 1; break; }
  }

  /* sort descending (selection sort on indices; n is small) */
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  for (int64_t i = 0; i < n; ++i) {
    int64_t best = i;
    for (int64_t j = i + 1; j < n; ++j)
      if (A[idx[j] * n + idx[j]] > A[idx[best] * n + idx[best]]) best = j;
    int64_t tmp = idx[i]; idx[i] = idx[best]; idx[best] = tmp;
  }
  for (int64_t j = 0; j < n; ++j) {
    const int64_t src = idx[j];
    evals[j] = A[src * n + src];
    /* sign: largest-magnitude entry positive, lowest row on ties */
    int64_t imax = 0;
    for (int64_t i = 1; i < n; ++i)
      if (fabs(Q[i * n + src]) > fabs(Q[imax * n + src])) imax = i;
    const double sg = (Q[imax * n + src] < 0.0) ? -1.0 : 1.0;
    for (int64_t i = 0; i < n; ++i) V[i * n + j] = sg * Q[i * n + src];
  }
  free(idx);
  free(A);
  free(Q);
  return converged ? sweeps : -1;
}

/* Leading K eigenvectors of W (n x n) -> F (n x K row-major). */
static int topk_eigvecs(int64_t n, const double* W, int64_t K, double* F, double* evals_out) {
  double* ev = (double*)malloc(sizeof(double) * (size_t)n);
  double* V = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int rc = orc_jacobi_eig(n, W, ev, V);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k < K; ++k) F[i * K + k] = V[i * n + k];
  if (evals_out)
    for (int64_t k = 0; k < n; ++k) evals_out[k] = ev[k];
  free(ev);
  free(V);
  return rc;
}

/* ---------------------------------------------------------------------------
 * TTM-chain helpers.  The first product may read a float tensor.
 * ------------------------------------------------------------------------- */
typedef struct {
  int N;
  int64_t dims[16];
  double* data; /* owned */
} otensor;

static int64_t numel(const int64_t* d, int N) { return prod_range(d, 0, N); }

/* Y = X x_j F^T, X given either as double (xd) or float (xf). */
static void chain_step(int N, int64_t* dims, const double* xd, const float* xf,
                       int j, const double* F, int64_t Kj, double** out) {
  double* Ft = transpose_factor(F, dims[j], Kj);
  int64_t nd[16];
  memcpy(nd, dims, sizeof(int64_t) * (size_t)N);
  nd[j] = Kj;
  double* Y = (double*)malloc(sizeof(double) * (size_t)numel(nd, N));
  if (xd) orc_ttm_d(N, dims, xd, j, Ft, Kj, Y);
  else orc_ttm_f(N, dims, xf, j, Ft, Kj, Y);
  free(Ft);
  dims[j] = Kj;
  *out = Y;
}

/* T x_{j in modes} F_j^T in the given order; returns a new buffer and its dims. */
static double* ttm_chain(int N, const int64_t* L, const double* Td, const float* Tf,
                         const double* const* F, const int64_t* K,
                         const int* order, int norder, int64_t* dims_out) {
  int64_t dims[16];
  memcpy(dims, L, sizeof(int64_t) * (size_t)N);
  double* cur = NULL;
  if (norder == 0) {
    int64_t n = numel(dims, N);
    cur = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) cur[i] = Td ? Td[i] : (double)Tf[i];
  }
  for (int s = 0; s < norder; ++s) {
    const int j = order[s];
    double* nxt = NULL;
    if (cur == NULL) chain_step(N, dims, Td, Tf, j, F[j], K[j], &nxt);
    else chain_step(N, dims, cur, NULL, j, F[j], K[j], &nxt);
    free(cur);
    cur = nxt;
  }
  memcpy(dims_out, dims, sizeof(int64_t) * (size_t)N);
  return cur;
}

/* ---------------------------------------------------------------------------
 * Fig. 2: one HOOI invocation.  t_is_float selects the storage of T.
 * F_in / F_out: arrays of N pointers to L_n x K_n row-major factors.
 * G_out: K_0 x ... x K_{N-1}.  gauss_seidel != 0 uses F_out[j] for j < n
 * (cross-check variant only).  Returns the worst Jacobi return code.
 * ------------------------------------------------------------------------- */
int orc_hooi_sweep(int N, const int64_t* L, const int64_t* K, const void* T, int t_is_float,
                   const double* const* F_in, double* const* F_out, double* G_out,
                   int gauss_seidel) {
  const double* Td = t_is_float ? NULL : (const double*)T;
  const float* Tf = t_is_float ? (const float*)T : NULL;
  const double* Fuse[16];
  int rc_all = 0;
  for (int n = 0; n < N; ++n) {
    int order[16], no = 0;
    for (int j = 0; j < N; ++j) {
      Fuse[j] = (gauss_seidel && j < n) ? F_out[j] : F_in[j];
      if (j != n) order[no++] = j;
    }
    int64_t dims[16];
    double* Z = ttm_chain(N, L, Td, Tf, Fuse, K, order, no, dims);
    double* W = (double*)malloc(sizeof(double) * (size_t)(L[n] * L[n]));
    orc_gram(N, dims, Z, n, W);
    int rc = topk_eigvecs(L[n], W, K[n], F_out[n], NULL);
    if (rc < 0) rc_all = -1;
    free(W);
    free(Z);
  }
  if (G_out) {
    int order[16];
    for (int j = 0; j < N; ++j) order[j] = j;
    int64_t dims[16];
    double* G = ttm_chain(N, L, Td, Tf, (const double* const*)F_out, K, order, N, dims);
    memcpy(G_out, G, sizeof(double) * (size_t)numel(K, N));
    free(G);
  }
  return rc_all;
}

/* Fig. 2 "New core": G = T x_1 F_1^T ... x_N F_N^T (natural order). */
void orc_core(int N, const int64_t* L, const int64_t* K, const void* T, int t_is_float,
              const double* const* F, double* G_out) {
  int order[16];
  for (int j = 0; j < N; ++j) order[j] = j;
  int64_t dims[16];
  double* G = ttm_chain(N, L, t_is_float ? NULL : (const double*)T,
                        t_is_float ? (const float*)T : NULL, F, K, order, N, dims);
  memcpy(G_out, G, sizeof(double) * (size_t)numel(K, N));
  free(G);
}

/* STHOSVD with the modes taken in the order order[0..N-1] (a permutation of
 * 0..N-1): Y <- T; for n = order[0], order[1], ...: F_n <- top-K_n eigvecs
 * of Y_(n) Y_(n)^T; Y <- Y x_n F_n^T.  G <- Y (modes keep their positions,
 * so G is K_0 x ... x K_{N-1} whatever the order).  evals_out (optional)
 * receives, for each mode n at offset L_0 + ... + L_{n-1}, all L_n
 * eigenvalues of the Gram that mode n's factor came from.  Returns -2 when
 * order is not a permutation. */
int orc_sthosvd_order(int N, const int64_t* L, const int64_t* K, const void* T, int t_is_float,
                      const int* order, double* const* F_out, double* G_out, double* evals_out) {
  int seen[16] = {0};
  for (int i = 0; i < N; ++i) {
    if (order[i] < 0 || order[i] >= N || seen[order[i]]) return -2;
    seen[order[i]] = 1;
  }
  int64_t dims[16];
  memcpy(dims, L, sizeof(int64_t) * (size_t)N);
  const int64_t n0 = numel(dims, N);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n0);
  for (int64_t i = 0; i < n0; ++i)
    Y[i] = t_is_float ? (double)((const float*)T)[i] : ((const double*)T)[i];
  int rc_all = 0;
  for (int i = 0; i < N; ++i) {
    const int n = order[i];
    double* W = (double*)malloc(sizeof(double) * (size_t)(dims[n] * dims[n]));
    orc_gram(N, dims, Y, n, W);
    double* ev = NULL;
    if (evals_out) ev = evals_out + len_sum(L, n);
    int rc = topk_eigvecs(dims[n], W, K[n], F_out[n], ev);
    if (rc < 0) rc_all = -1;
    free(W);
    double* nxt = NULL;
    chain_step(N, dims, Y, NULL, n, F_out[n], K[n], &nxt);
    free(Y);
    Y = nxt;
  }
  memcpy(G_out, Y, sizeof(double) * (size_t)numel(K, N));
  free(Y);
  return rc_all;
}

/* STHOSVD in natural mode order 0, 1, ..., N-1. */
int orc_sthosvd(int N, const int64_t* L, const int64_t* K, const void* T, int t_is_float,
                double* const* F_out, double* G_out, double* evals_out) {
  int order[16];
  for (int n = 0; n < N; ++n) order[n] = n;
  return orc_sthosvd_order(N, L, K, T, t_is_float, order, F_out, G_out, evals_out);
}

/* Sum of squares in double. */
double orc_norm2_d(int64_t n, const double* x) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += x[i] * x[i];
  return s;
}

double orc_norm2_f(int64_t n, const float* x) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += (double)x[i] * (double)x[i];
  return s;
}

/* Sec. 2.2 error metric via the orthonormal-factor identity. */
double orc_fit(double normT2, double normG2) {
  double r2 = normT2 - normG2;
  if (r2 < 0.0) r2 = 0.0;
  return 1.0 - sqrt(r2) / sqrt(normT2);
}

/* Reconstruction Z = G x_1 F_1 ... x_N F_N (Sec. 2.2), written to Xhat. */
void orc_reconstruct(int N, const int64_t* L, const int64_t* K, const double* G,
                     const double* const* F, double* Xhat) {
  int64_t dims[16];
  memcpy(dims, K, sizeof(int64_t) * (size_t)N);
  int64_t n0 = numel(dims, N);
  double* cur = (double*)malloc(sizeof(double) * (size_t)n0);
  memcpy(cur, G, sizeof(double) * (size_t)n0);
  for (int j = 0; j < N; ++j) {
    /* x_j F_j with F_j of size L_j x K_j: A = F_j directly */
    int64_t nd[16];
    memcpy(nd, dims, sizeof(int64_t) * (size_t)N);
    nd[j] = L[j];
    double* nxt = (double*)malloc(sizeof(double) * (size_t)numel(nd, N));
    orc_ttm_d(N, dims, cur, j, F[j], L[j], nxt);
    free(cur);
    cur = nxt;
    dims[j] = L[j];
  }
  memcpy(Xhat, cur, sizeof(double) * (size_t)numel(L, N));
  free(cur);
}

/* Direct error ||T - G x F||_F (Sec. 2.2), no identity used. */
double orc_residual(int N, const int64_t* L, const int64_t* K, const void* T, int t_is_float,
                    const double* G, const double* const* F) {
  const int64_t n0 = numel(L, N);
  double* Xh = (double*)malloc(sizeof(double) * (size_t)n0);
  orc_reconstruct(N, L, K, G, F, Xh);
  double s = 0.0;
  for (int64_t i = 0; i < n0; ++i) {
    const double t = t_is_float ? (double)((const float*)T)[i] : ((const double*)T)[i];
    const double d = t - Xh[i];
    s += d * d;
  }
  free(Xh);
  return sqrt(s);
}
