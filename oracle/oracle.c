/*
 * oracle.c -- plain, slow FP64 CPU oracle for the SRTM filter and smoother of
 * "Parallel state estimation for systems with integrated measurements"
 * (Yaghoobi & Sarkka, arXiv 2410.00627).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: only the test-suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA path.  Every routine below follows the paper's equations in
 * the paper's order with plain loops; nothing is blocked, fused or reordered
 * beyond the algebra stated at each routine.
 *
 * Conventions (the readings of the paper that this oracle takes):
 *   - Matrices are row-major double arrays.  A is the paper's fast transition
 *     (called F at the library boundary).
 *   - H multiplies the SUM of the l fast states of an interval, so the
 *     paper's C/l equals H (Sec. III, Eq. (5b)/(6b): C relates the average).
 *   - Q~ = E[w_bar w_bar^T] = blockdiag(Q, ..., Q) (white fast noise, Eq. (9)).
 *   - Interval k (paper, 1-based) has fast states x_{k,1..l}; x_{k,0}=x_{k-1,l},
 *     x_{0,l}=x_0 ~ N(m0,P0).  Arrays here use 0-based k.
 *   - Parallel IMKF element for k=1 has eta_1=0, J_1=0 (Sec. IV: only F_1, d_1,
 *     D_1 are given; a_1 is always the leftmost operand).
 *   - Parallel IMS element: S_k = P^f_{k,1} - E_k A (P^f_{k,1,l})^T.  The
 *     printed formula omits the transpose; with it, S_k equals
 *     P^f_{k,1} - E_k P^-_{k+1,1} E_k^T (the covariance of x_{k,1} given
 *     x_{k+1,1}), which is what Lemma-9-style conditioning gives.  Flag bit
 *     ORACLE_LITERAL_SK selects the printed (untransposed) reading, kept only
 *     so that a test can show the brute-force pin rejects it.
 *
 * Parity status: every exported function is pinned by the test-suite against
 * a brute-force joint-Gaussian posterior, the textbook Kalman/RTS case l=1,
 * the discrete algebraic Riccati equation and internal equivalences.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_LITERAL_SK 1

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                        */
/* ------------------------------------------------------------------------ */

/* C (r x c) = alpha * op(A) op(B) + beta * C.  op(A) is r x k, op(B) is k x c.
 * tA: A is stored k x r and used transposed; tB: B is stored c x k.
 * C must not alias A or B. */
static void gemm(int r, int k, int c, double alpha, const double *A, int tA,
                 const double *B, int tB, double beta, double *C) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double s = 0.0;
      for (int p = 0; p < k; ++p) {
        double a = tA ? A[p * r + i] : A[i * k + p];
        double b = tB ? B[j * k + p] : B[p * c + j];
        s += a * b;
      }
      C[i * c + j] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[i * c + j]);
    }
}

static void copy(int n, const double *a, double *b) { memcpy(b, a, sizeof(double) * (size_t)n); }
static void axpy(int n, double alpha, const double *x, double *y) {
  for (int i = 0; i < n; ++i) y[i] += alpha * x[i];
}
static void eye(int n, double *I) {
  memset(I, 0, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
}
static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* Solve M X = B in place (M n x n, B n x nrhs) by Gaussian elimination with
 * partial pivoting on a copy of M.  Returns 0, or -1 if M is singular. */
static int solve(int n, const double *M, int nrhs, double *B) {
  double *a = dalloc((size_t)n * n);
  copy(n * n, M, a);
  int rc = 0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r * n + col]) > fabs(a[piv * n + col])) piv = r;
    if (a[piv * n + col] == 0.0) { rc = -1; break; }
    if (piv != col) {
      for (int j = 0; j < n; ++j) { double t = a[col * n + j]; a[col * n + j] = a[piv * n + j]; a[piv * n + j] = t; }
      for (int j = 0; j < nrhs; ++j) { double t = B[col * nrhs + j]; B[col * nrhs + j] = B[piv * nrhs + j]; B[piv * nrhs + j] = t; }
    }
    for (int r = col + 1; r < n; ++r) {
      double f = a[r * n + col] / a[col * n + col];
      if (f == 0.0) continue;
      for (int j = col; j < n; ++j) a[r * n + j] -= f * a[col * n + j];
      for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= f * B[col * nrhs + j];
    }
  }
  if (rc == 0)
    for (int col = n - 1; col >= 0; --col)
      for (int j = 0; j < nrhs; ++j) {
        double s = B[col * nrhs + j];
        for (int p = col + 1; p < n; ++p) s -= a[col * n + p] * B[p * nrhs + j];
        B[col * nrhs + j] = s / a[col * n + col];
      }
  free(a);
  return rc;
}

/* Minv = M^{-1} (n x n). */
static int inverse(int n, const double *M, double *Minv) {
  eye(n, Minv);
  return solve(n, M, n, Minv);
}

/* X (r x n) = B M^{-1}:  solve M^T X^T = B^T. */
static int right_solve(int n, const double *M, int r, const double *B, double *X) {
  double *Mt = dalloc((size_t)n * n), *Bt = dalloc((size_t)n * r);
  for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) Mt[i * n + j] = M[j * n + i];
  for (int i = 0; i < r; ++i) for (int j = 0; j < n; ++j) Bt[j * r + i] = B[i * n + j];
  int rc = solve(n, Mt, r, Bt);
  for (int i = 0; i < r; ++i) for (int j = 0; j < n; ++j) X[i * n + j] = Bt[j * r + i];
  free(Mt); free(Bt);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* model constants of Sec. III                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n, m, l;
  double *Apow;   /* (l+1) x n x n : A^0 .. A^l                                   */
  double *Abar;   /* A^l                                          (Eq. 7)          */
  double *Qbar;   /* G_bar Q~ G_bar^T                             (Eq. 9)          */
  double *Cbar;   /* (C/l) sum_{i=1..l} A^i = H sum A^i   (m x n) (Eq. 10)        */
  double *MQM;    /* M_bar Q~ M_bar^T                     (m x m) (Eq. 11,12)      */
  double *GQM;    /* G_bar Q~ M_bar^T                     (n x m) (Eq. 11,12)      */
  double *GQG;    /* script-G Q~ script-G^T            (ln x ln) (Eq. 14,15)     */
  double *AtHt;   /* script-A^T script-H^T                (n x m) (Eq. 14,16)     */
  double *GQGHt;  /* script-G Q~ script-G^T script-H^T   (ln x m) (Eq. 15,16)     */
  int nu;         /* inputs (0: none)                                               */
  double *B;      /* B                                    (n x nu)                 */
  double *Bbar;   /* B_bar = [A^{l-1}B ... AB B]          (n x l nu) (Eq. 7)       */
  double *Dbar;   /* D_bar = (C/l)[sum_{i<l}A^i B, ..., B] (m x l nu) (Eq. 10)     */
  double *sB;     /* stacked fast input map, block (i,j) = A^{i-j} B, j <= i
                     (ln x l nu): the input part of the stacked means (Eq. 13)    */
} model_t;

static void model_free(model_t *M) {
  free(M->Apow); free(M->Abar); free(M->Qbar); free(M->Cbar); free(M->MQM);
  free(M->GQM); free(M->GQG); free(M->AtHt); free(M->GQGHt);
  free(M->B); free(M->Bbar); free(M->Dbar); free(M->sB);
}

/* The input matrices of the lifted and stacked models (nu > 0): the
 * interval's inputs are u_bar_k = [u_{k-1,l}; u_{k,1}; ...; u_{k,l-1}], the
 * inputs that drive x_{k,1}, ..., x_{k,l}. */
static void model_inputs(model_t *M, int nu, const double *B, const double *H) {
  int n = M->n, m = M->m, l = M->l, ln = l * n, lu = l * nu;
  M->nu = nu;
  M->B = M->Bbar = M->Dbar = M->sB = NULL;
  if (nu <= 0 || !B) { M->nu = 0; return; }
  M->B = dalloc((size_t)n * nu);
  copy(n * nu, B, M->B);
  M->Bbar = dalloc((size_t)n * lu);
  M->Dbar = dalloc((size_t)m * lu);
  M->sB = dalloc((size_t)ln * lu);
  double *AB = dalloc((size_t)(l + 1) * n * nu), *SB = dalloc((size_t)n * nu), *HSB = dalloc((size_t)m * nu);
  for (int i = 0; i <= l; ++i) gemm(n, n, nu, 1.0, M->Apow + (size_t)i * n * n, 0, B, 0, 0.0, AB + (size_t)i * n * nu);
  for (int j = 0; j < l; ++j) {
    /* Bbar block j = A^{l-1-j} B;  Dbar block j = H sum_{i=0}^{l-1-j} A^i B */
    const double *Ab = AB + (size_t)(l - 1 - j) * n * nu;
    for (int r = 0; r < n; ++r) for (int c = 0; c < nu; ++c) M->Bbar[r * lu + j * nu + c] = Ab[r * nu + c];
    memset(SB, 0, sizeof(double) * (size_t)n * nu);
    for (int i = 0; i <= l - 1 - j; ++i) axpy(n * nu, 1.0, AB + (size_t)i * n * nu, SB);
    gemm(m, n, nu, 1.0, H, 0, SB, 0, 0.0, HSB);
    for (int r = 0; r < m; ++r) for (int c = 0; c < nu; ++c) M->Dbar[r * lu + j * nu + c] = HSB[r * nu + c];
  }
  /* stacked: block (i,j) = A^{i-j} B for j <= i (x_{k,i+1} gets u_{k,j}) */
  for (int i = 0; i < l; ++i)
    for (int j = 0; j <= i; ++j) {
      const double *Ab = AB + (size_t)(i - j) * n * nu;
      for (int r = 0; r < n; ++r) for (int c = 0; c < nu; ++c) M->sB[(size_t)(i * n + r) * lu + j * nu + c] = Ab[r * nu + c];
    }
  free(AB); free(SB); free(HSB);
}

/* Forms the lifted matrices literally: G_bar = [A^{l-1} ... A I] (n x ln),
 * Q~ = blockdiag(Q) (ln x ln), M_bar = (C/l)[sum_{i<l}A^i, sum_{i<l-1}A^i, ..., I]
 * (m x ln), script-G = block lower-triangular with blocks A^{i-j} (ln x ln),
 * script-H = (1/l)[C ... C] = [H ... H] (m x ln). */
static void model_build(model_t *M, int n, int m, int l, const double *A,
                        const double *Q, const double *H) {
  int ln = l * n;
  M->n = n; M->m = m; M->l = l;
  M->Apow = dalloc((size_t)(l + 1) * n * n);
  eye(n, M->Apow);
  for (int i = 1; i <= l; ++i)
    gemm(n, n, n, 1.0, M->Apow + (size_t)(i - 1) * n * n, 0, A, 0, 0.0, M->Apow + (size_t)i * n * n);
  M->Abar = dalloc((size_t)n * n);
  copy(n * n, M->Apow + (size_t)l * n * n, M->Abar);

  double *Gbar = dalloc((size_t)n * ln);     /* block j (0-based) = A^{l-1-j} */
  double *Qt = dalloc((size_t)ln * ln);      /* blockdiag(Q) */
  double *Mbar = dalloc((size_t)m * ln);     /* block j = H * sum_{i=0}^{l-1-j} A^i */
  for (int j = 0; j < l; ++j) {
    const double *Ap = M->Apow + (size_t)(l - 1 - j) * n * n;
    for (int r = 0; r < n; ++r) for (int c = 0; c < n; ++c) Gbar[r * ln + j * n + c] = Ap[r * n + c];
    for (int r = 0; r < n; ++r) for (int c = 0; c < n; ++c) Qt[(size_t)(j * n + r) * ln + j * n + c] = Q[r * n + c];
    double *Ssum = dalloc((size_t)n * n);
    for (int i = 0; i <= l - 1 - j; ++i) axpy(n * n, 1.0, M->Apow + (size_t)i * n * n, Ssum);
    double *HS = dalloc((size_t)m * n);
    gemm(m, n, n, 1.0, H, 0, Ssum, 0, 0.0, HS);
    for (int r = 0; r < m; ++r) for (int c = 0; c < n; ++c) Mbar[r * ln + j * n + c] = HS[r * n + c];
    free(Ssum); free(HS);
  }
  double *GQ = dalloc((size_t)n * ln), *MQ = dalloc((size_t)m * ln);
  gemm(n, ln, ln, 1.0, Gbar, 0, Qt, 0, 0.0, GQ);
  gemm(m, ln, ln, 1.0, Mbar, 0, Qt, 0, 0.0, MQ);
  M->Qbar = dalloc((size_t)n * n);
  gemm(n, ln, n, 1.0, GQ, 0, Gbar, 1, 0.0, M->Qbar);
  M->GQM = dalloc((size_t)n * m);
  gemm(n, ln, m, 1.0, GQ, 0, Mbar, 1, 0.0, M->GQM);
  M->MQM = dalloc((size_t)m * m);
  gemm(m, ln, m, 1.0, MQ, 0, Mbar, 1, 0.0, M->MQM);
  double *Asum = dalloc((size_t)n * n);
  for (int i = 1; i <= l; ++i) axpy(n * n, 1.0, M->Apow + (size_t)i * n * n, Asum);
  M->Cbar = dalloc((size_t)m * n);
  gemm(m, n, n, 1.0, H, 0, Asum, 0, 0.0, M->Cbar);

  /* stacked fast model of Eq. (13)-(16) */
  double *sG = dalloc((size_t)ln * ln);
  for (int i = 0; i < l; ++i)
    for (int j = 0; j <= i; ++j) {
      const double *Ap = M->Apow + (size_t)(i - j) * n * n;
      for (int r = 0; r < n; ++r) for (int c = 0; c < n; ++c) sG[(size_t)(i * n + r) * ln + j * n + c] = Ap[r * n + c];
    }
  double *sGQ = dalloc((size_t)ln * ln);
  gemm(ln, ln, ln, 1.0, sG, 0, Qt, 0, 0.0, sGQ);
  M->GQG = dalloc((size_t)ln * ln);
  gemm(ln, ln, ln, 1.0, sGQ, 0, sG, 1, 0.0, M->GQG);
  double *sH = dalloc((size_t)m * ln);
  for (int j = 0; j < l; ++j) for (int r = 0; r < m; ++r) for (int c = 0; c < n; ++c) sH[r * ln + j * n + c] = H[r * n + c];
  double *sA = dalloc((size_t)ln * n);
  for (int i = 0; i < l; ++i) {
    const double *Ap = M->Apow + (size_t)(i + 1) * n * n;
    for (int r = 0; r < n; ++r) for (int c = 0; c < n; ++c) sA[(size_t)(i * n + r) * n + c] = Ap[r * n + c];
  }
  M->AtHt = dalloc((size_t)n * m);
  gemm(n, ln, m, 1.0, sA, 1, sH, 1, 0.0, M->AtHt);
  M->GQGHt = dalloc((size_t)ln * m);
  gemm(ln, ln, m, 1.0, M->GQG, 0, sH, 1, 0.0, M->GQGHt);

  free(Gbar); free(Qt); free(Mbar); free(GQ); free(MQ); free(Asum);
  free(sG); free(sGQ); free(sH); free(sA);
}

/* ------------------------------------------------------------------------ */
/* Sec. III-A: sequential IMKF for the slow states x_{k,l}, Eq. (9),(12)     */
/* ------------------------------------------------------------------------ */

/* One IMKF step from (mp,Pp) = p(x_{k-1,l}|y_{1:k-1}) with measurement yk. */
/* log|det S| of a symmetric positive definite S (m x m) by the Cholesky
 * factor S = G G^T: 2 sum_j log G_jj.  Returns -1 if S is not positive definite. */
static int logdet_spd(int m, const double *S, double *out) {
  double *G = dalloc((size_t)m * m);
  int rc = 0;
  double acc = 0.0;
  for (int j = 0; j < m && !rc; ++j) {
    double d = S[j * m + j];
    for (int k = 0; k < j; ++k) d -= G[j * m + k] * G[j * m + k];
    if (!(d > 0.0)) { rc = -1; break; }
    G[j * m + j] = sqrt(d);
    acc += log(G[j * m + j]);
    for (int i = j + 1; i < m; ++i) {
      double v = S[i * m + j];
      for (int k = 0; k < j; ++k) v -= G[i * m + k] * G[j * m + k];
      G[i * m + j] = v / G[j * m + j];
    }
  }
  *out = 2.0 * acc;
  free(G);
  return rc;
}

/* One step of the slow-rate IMKF, Eq. (9)-(12).  term (optional): the
 * measurement's log predictive density log N(y_k; C_bar m_{k-1}, S_k), the
 * k-th term of the prediction-error decomposition of log p(y_{1:N}). */
static int imkf_step(const model_t *M, const double *R, const double *mp, const double *Pp,
                     const double *yk, double *mf, double *Pf, double *term, const double *uk) {
  int n = M->n, m = M->m, rc = 0;
  double *mminus = dalloc(n), *Pminus = dalloc((size_t)n * n), *AP = dalloc((size_t)n * n);
  double *cross = dalloc((size_t)n * m), *S = dalloc((size_t)m * m), *CP = dalloc((size_t)m * n);
  double *L = dalloc((size_t)n * m), *innov = dalloc(m);
  gemm(n, n, 1, 1.0, M->Abar, 0, mp, 0, 0.0, mminus);                /* m^- = A_bar m      */
  if (M->nu && uk) gemm(n, M->l * M->nu, 1, 1.0, M->Bbar, 0, uk, 0, 1.0, mminus); /* + B_bar u_bar_k */
  gemm(n, n, n, 1.0, M->Abar, 0, Pp, 0, 0.0, AP);
  gemm(n, n, n, 1.0, AP, 0, M->Abar, 1, 0.0, Pminus);                /* A_bar P A_bar^T    */
  axpy(n * n, 1.0, M->Qbar, Pminus);                                 /*   + Q_bar          */
  gemm(n, n, m, 1.0, AP, 0, M->Cbar, 1, 0.0, cross);                 /* A_bar P C_bar^T    */
  axpy(n * m, 1.0, M->GQM, cross);                                   /*   + G Q~ M^T       */
  gemm(m, n, n, 1.0, M->Cbar, 0, Pp, 0, 0.0, CP);
  gemm(m, n, m, 1.0, CP, 0, M->Cbar, 1, 0.0, S);                     /* C_bar P C_bar^T    */
  axpy(m * m, 1.0, M->MQM, S);                                       /*   + M Q~ M^T       */
  axpy(m * m, 1.0, R, S);                                            /*   + R              */
  if (right_solve(m, S, n, cross, L)) rc = -1;                       /* L_k                */
  gemm(m, n, 1, -1.0, M->Cbar, 0, mp, 0, 0.0, innov);
  axpy(m, 1.0, yk, innov);                                           /* y - C_bar m        */
  if (M->nu && uk) gemm(m, M->l * M->nu, 1, -1.0, M->Dbar, 0, uk, 0, 1.0, innov);   /* - D_bar u_bar_k */
  if (term) {  /* -1/2 (m log 2 pi + log det S + innov^T S^-1 innov) */
    double *z = dalloc(m), ld = 0.0, q = 0.0;
    copy(m, innov, z);
    if (solve(m, S, 1, z) || logdet_spd(m, S, &ld)) rc = -1;
    for (int j = 0; j < m; ++j) q += innov[j] * z[j];
    *term = -0.5 * (m * log(2.0 * 3.14159265358979323846) + ld + q);
    free(z);
  }
  copy(n, mminus, mf);
  gemm(n, m, 1, 1.0, L, 0, innov, 0, 1.0, mf);
  copy(n * n, Pminus, Pf);
  gemm(n, m, n, -1.0, L, 0, cross, 1, 1.0, Pf);                      /* P^- - L cross^T    */
  /* The update above is symmetric in exact arithmetic, but in floating point
   * its antisymmetric roundoff is propagated by a map that is not a
   * contraction (it grows ~2.5x per step on the 4-species chain), so the
   * recursion would diverge after ~50 steps.  Replace P^f by its symmetric
   * part, which leaves the exact result unchanged. */
  for (int r = 0; r < n; ++r)
    for (int c = r + 1; c < n; ++c) {
      double v = 0.5 * (Pf[r * n + c] + Pf[c * n + r]);
      Pf[r * n + c] = v; Pf[c * n + r] = v;
    }
  free(mminus); free(Pminus); free(AP); free(cross); free(S); free(CP); free(L); free(innov);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-B: fast-rate filter of one interval, Eq. (15)-(17), on the       */
/* blocks of Remark 2.                                                        */
/* ------------------------------------------------------------------------ */


/* block (bi,bj) of an (l n x l n) row-major matrix */
static void get_block(int n, int ln, const double *X, int bi, int bj, double *out) {
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) out[r * n + c] = X[(size_t)(bi * n + r) * ln + bj * n + c];
}

/* Given (mp,Pp) = p(x_{k-1,l}|y_{1:k-1}) and y_k, returns for i=1..l (array index i-1):
 *   mf [i] = m^f_{k,i}     (l x n)
 *   Pii[i] = P^f_{k,i,i}   (l x n x n)
 *   Pil[i] = P^f_{k,i,l}   (l x n x n)
 * Eq. (15)-(17) written blockwise (script-H = [H ... H]):
 *   M^-_i        = A^i m
 *   (P^- H^T)_i  = A^i P (script-A^T script-H^T) + (script-G Q~ script-G^T script-H^T)_i
 *   S            = script-H P^- script-H^T + R = sum_i H (P^- H^T)_i + R
 *   L_i          = (P^- H^T)_i S^{-1}
 *   m^f_i        = M^-_i + L_i (y - sum_j H A^j m)
 *   P^-_{ij}     = A^i P A^{jT} + (script-G Q~ script-G^T)_{ij}
 *   P^f_{ij}     = P^-_{ij} - L_i (P^- H^T)_j^T                                 */
static int fast_filter_interval(const model_t *M, const double *H, const double *R,
                                const double *mp, const double *Pp, const double *yk,
                                double *mf, double *Pii, double *Pil, const double *uk) {
  int n = M->n, m = M->m, l = M->l, ln = l * n, rc = 0;
  double *sBu = dalloc((size_t)ln);   /* input part of the stacked means */
  if (M->nu && uk) gemm(ln, l * M->nu, 1, 1.0, M->sB, 0, uk, 0, 0.0, sBu);
  double *PHt = dalloc((size_t)ln * m), *S = dalloc((size_t)m * m), *L = dalloc((size_t)ln * m);
  double *PAtHt = dalloc((size_t)n * m), *innov = dalloc(m), *Am = dalloc(n);
  double *AP = dalloc((size_t)n * n), *blk = dalloc((size_t)n * n);
  gemm(n, n, m, 1.0, Pp, 0, M->AtHt, 0, 0.0, PAtHt);
  for (int i = 0; i < l; ++i) {
    gemm(n, n, m, 1.0, M->Apow + (size_t)(i + 1) * n * n, 0, PAtHt, 0, 0.0, PHt + (size_t)i * n * m);
    axpy(n * m, 1.0, M->GQGHt + (size_t)i * n * m, PHt + (size_t)i * n * m);
  }
  copy(m * m, R, S);
  for (int i = 0; i < l; ++i) gemm(m, n, m, 1.0, H, 0, PHt + (size_t)i * n * m, 0, 1.0, S);
  if (right_solve(m, S, ln, PHt, L)) rc = -1;
  copy(m, yk, innov);
  for (int i = 0; i < l; ++i) {
    gemm(n, n, 1, 1.0, M->Apow + (size_t)(i + 1) * n * n, 0, mp, 0, 0.0, Am);
    axpy(n, 1.0, sBu + (size_t)i * n, Am);
    gemm(m, n, 1, -1.0, H, 0, Am, 0, 1.0, innov);
  }
  for (int i = 0; i < l; ++i) {
    const double *Ai = M->Apow + (size_t)(i + 1) * n * n;
    const double *Li = L + (size_t)i * n * m;
    gemm(n, n, 1, 1.0, Ai, 0, mp, 0, 0.0, mf + (size_t)i * n);
    axpy(n, 1.0, sBu + (size_t)i * n, mf + (size_t)i * n);
    gemm(n, m, 1, 1.0, Li, 0, innov, 0, 1.0, mf + (size_t)i * n);
    gemm(n, n, n, 1.0, Ai, 0, Pp, 0, 0.0, AP);
    /* (i,i) block */
    double *Po = Pii + (size_t)i * n * n;
    gemm(n, n, n, 1.0, AP, 0, Ai, 1, 0.0, Po);
    get_block(n, ln, M->GQG, i, i, blk);
    axpy(n * n, 1.0, blk, Po);
    gemm(n, m, n, -1.0, Li, 0, PHt + (size_t)i * n * m, 1, 1.0, Po);
    /* (i,l) block */
    Po = Pil + (size_t)i * n * n;
    gemm(n, n, n, 1.0, AP, 0, M->Apow + (size_t)l * n * n, 1, 0.0, Po);
    get_block(n, ln, M->GQG, i, l - 1, blk);
    axpy(n * n, 1.0, blk, Po);
    gemm(n, m, n, -1.0, Li, 0, PHt + (size_t)(l - 1) * n * m, 1, 1.0, Po);
  }
  free(PHt); free(S); free(L); free(PAtHt); free(innov); free(Am); free(AP); free(blk); free(sBu);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-C: the sequential SRTM smoother, Eq. (21),(22)                    */
/* ------------------------------------------------------------------------ */

/* Smoothing step shared by Eq. (21) (all fast states) and Eq. (22) (first
 * state): given the filtered quantities of interval k and p(x_{k+1,1}|y_{1:N}),
 *   P^-_{k+1,1} = A P^f_{k,l,l} A^T + Q,   m^-_{k+1,1} = A m^f_{k,l} + B u_{k,l}
 *   G_{k,i}     = P^f_{k,i,l} A^T [P^-_{k+1,1}]^{-1}
 *   m^s_{k,i}   = m^f_{k,i} + G_{k,i} (m^s_{k+1,1} - m^-_{k+1,1})
 *   P^s_{k,i,i} = P^f_{k,i,i} + G_{k,i} (P^s_{k+1,1} - P^-_{k+1,1}) G_{k,i}^T */
static int smooth_step(int n, const double *A, const double *Q, const double *ml,
                       const double *Pll, const double *mfi, const double *Pfii,
                       const double *Pfil, const double *ms_next, const double *Ps_next,
                       double *ms, double *Ps, const double *bnext) {
  double *AP = dalloc((size_t)n * n), *Pm = dalloc((size_t)n * n), *mm = dalloc(n);
  double *PA = dalloc((size_t)n * n), *G = dalloc((size_t)n * n), *dm = dalloc(n);
  double *dP = dalloc((size_t)n * n), *GdP = dalloc((size_t)n * n);
  int rc = 0;
  gemm(n, n, n, 1.0, A, 0, Pll, 0, 0.0, AP);
  gemm(n, n, n, 1.0, AP, 0, A, 1, 0.0, Pm);
  axpy(n * n, 1.0, Q, Pm);
  gemm(n, n, 1, 1.0, A, 0, ml, 0, 0.0, mm);
  if (bnext) axpy(n, 1.0, bnext, mm);                        /* + B u_{k+1,0} */
  gemm(n, n, n, 1.0, Pfil, 0, A, 1, 0.0, PA);
  if (right_solve(n, Pm, n, PA, G)) rc = -1;
  copy(n, ms_next, dm); axpy(n, -1.0, mm, dm);
  copy(n, mfi, ms);
  gemm(n, n, 1, 1.0, G, 0, dm, 0, 1.0, ms);
  copy(n * n, Ps_next, dP); axpy(n * n, -1.0, Pm, dP);
  gemm(n, n, n, 1.0, G, 0, dP, 0, 0.0, GdP);
  copy(n * n, Pfii, Ps);
  gemm(n, n, n, 1.0, GdP, 0, G, 1, 1.0, Ps);
  free(AP); free(Pm); free(mm); free(PA); free(G); free(dm); free(dP); free(GdP);
  return rc;
}

/* Inputs of interval k (0-based): u_bar = rows k l .. k l + l - 1 of u (NULL
 * without inputs); B u_{k+1,0} = B u_{(k+1) l}, the input term of the
 * prediction m^-_{k+1,1} in the smoother (NULL without inputs). */
#define UBAR(k) (M.nu ? u + (size_t)(k) * l * M.nu : NULL)
#define BNEXT(k) (M.nu ? (gemm(n, M.nu, 1, 1.0, M.B, 0, u + (size_t)((k) + 1) * l * M.nu, 0, 0.0, bnext), bnext) : NULL)

/* Sequential reference: IMKF (Eq. 9,12) for x_{k,l}; fast filter (Eq. 15-17);
 * sequential smoother for x_{k,1} (Eq. 22) and for all fast states (Eq. 21).
 * Arrays: y is N x m.  Every output may be NULL.  Fast outputs cover the
 * intervals k in [k_lo, k_hi) (0-based), row (k-k_lo)*l + (i-1) for x_{k+1,i}
 * in the paper's 1-based index.  Returns 0, or -1 if a solve was singular. */
int oracle_srtm_sequential(int n, int m, int l, int N, const double *A, const double *Q,
                           const double *H, const double *R, const double *m0,
                           const double *P0, const double *y, int k_lo, int k_hi,
                           double *slow_filt_mean, double *slow_filt_cov,
                           double *first_smooth_mean, double *first_smooth_cov,
                           double *fast_filt_mean, double *fast_filt_cov,
                           double *fast_smooth_mean, double *fast_smooth_cov, int nu, const double *B,
                           const double *u) {
  if (n < 1 || m < 1 || l < 1 || N < 1 || k_lo < 0 || k_hi > N || k_lo > k_hi) return -2;
  model_t M;
  model_build(&M, n, m, l, A, Q, H);
  model_inputs(&M, u ? nu : 0, B, H);
  int rc = 0, nn = n * n;
  double *bnext = dalloc(n);
  double *mfl = dalloc((size_t)N * n), *Pfl = dalloc((size_t)N * nn);
  /* IMKF */
  for (int k = 0; k < N; ++k) {
    const double *mp = k ? mfl + (size_t)(k - 1) * n : m0;
    const double *Pp = k ? Pfl + (size_t)(k - 1) * nn : P0;
    if (imkf_step(&M, R, mp, Pp, y + (size_t)k * m, mfl + (size_t)k * n, Pfl + (size_t)k * nn, NULL,
                  UBAR(k)))
      rc = -1;
  }
  if (slow_filt_mean) copy(N * n, mfl, slow_filt_mean);
  if (slow_filt_cov) copy(N * nn, Pfl, slow_filt_cov);

  int need_smooth = first_smooth_mean || first_smooth_cov || fast_smooth_mean || fast_smooth_cov;
  double *ms1 = NULL, *Ps1 = NULL;
  double *mf = dalloc((size_t)l * n), *Pii = dalloc((size_t)l * nn), *Pil = dalloc((size_t)l * nn);
  if (need_smooth) {
    double *m1 = dalloc((size_t)N * n), *P11 = dalloc((size_t)N * nn), *P1l = dalloc((size_t)N * nn);
    double *ml = dalloc((size_t)N * n), *Pll = dalloc((size_t)N * nn);
    for (int k = 0; k < N; ++k) {
      const double *mp = k ? mfl + (size_t)(k - 1) * n : m0;
      const double *Pp = k ? Pfl + (size_t)(k - 1) * nn : P0;
      if (fast_filter_interval(&M, H, R, mp, Pp, y + (size_t)k * m, mf, Pii, Pil, UBAR(k))) rc = -1;
      copy(n, mf, m1 + (size_t)k * n);
      copy(nn, Pii, P11 + (size_t)k * nn);
      copy(nn, Pil, P1l + (size_t)k * nn);
      copy(n, mf + (size_t)(l - 1) * n, ml + (size_t)k * n);
      copy(nn, Pii + (size_t)(l - 1) * nn, Pll + (size_t)k * nn);
    }
    ms1 = dalloc((size_t)N * n); Ps1 = dalloc((size_t)N * nn);
    copy(n, m1 + (size_t)(N - 1) * n, ms1 + (size_t)(N - 1) * n);
    copy(nn, P11 + (size_t)(N - 1) * nn, Ps1 + (size_t)(N - 1) * nn);
    for (int k = N - 2; k >= 0; --k)
      if (smooth_step(n, A, Q, ml + (size_t)k * n, Pll + (size_t)k * nn, m1 + (size_t)k * n,
                      P11 + (size_t)k * nn, P1l + (size_t)k * nn, ms1 + (size_t)(k + 1) * n,
                      Ps1 + (size_t)(k + 1) * nn, ms1 + (size_t)k * n, Ps1 + (size_t)k * nn, BNEXT(k)))
        rc = -1;
    if (first_smooth_mean) copy(N * n, ms1, first_smooth_mean);
    if (first_smooth_cov) copy(N * nn, Ps1, first_smooth_cov);
    free(m1); free(P11); free(P1l); free(ml); free(Pll);
  }
  if (fast_filt_mean || fast_filt_cov || fast_smooth_mean || fast_smooth_cov) {
    for (int k = k_lo; k < k_hi; ++k) {
      const double *mp = k ? mfl + (size_t)(k - 1) * n : m0;
      const double *Pp = k ? Pfl + (size_t)(k - 1) * nn : P0;
      if (fast_filter_interval(&M, H, R, mp, Pp, y + (size_t)k * m, mf, Pii, Pil, UBAR(k))) rc = -1;
      size_t row = (size_t)(k - k_lo) * l;
      if (fast_filt_mean) copy(l * n, mf, fast_filt_mean + row * n);
      if (fast_filt_cov) copy(l * nn, Pii, fast_filt_cov + row * nn);
      if (fast_smooth_mean || fast_smooth_cov) {
        for (int i = 0; i < l; ++i) {
          double *msi = dalloc(n), *Psi = dalloc(nn);
          if (k == N - 1) {   /* last interval: smoothed = filtered */
            copy(n, mf + (size_t)i * n, msi);
            copy(nn, Pii + (size_t)i * nn, Psi);
          } else if (smooth_step(n, A, Q, mf + (size_t)(l - 1) * n, Pii + (size_t)(l - 1) * nn,
                                 mf + (size_t)i * n, Pii + (size_t)i * nn, Pil + (size_t)i * nn,
                                 ms1 + (size_t)(k + 1) * n, Ps1 + (size_t)(k + 1) * nn, msi, Psi, BNEXT(k))) {
            rc = -1;
          }
          if (fast_smooth_mean) copy(n, msi, fast_smooth_mean + (row + i) * n);
          if (fast_smooth_cov) copy(nn, Psi, fast_smooth_cov + (row + i) * nn);
          free(msi); free(Psi);
        }
      }
    }
  }
  free(mf); free(Pii); free(Pil); free(ms1); free(Ps1); free(mfl); free(Pfl); free(bnext);
  model_free(&M);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. IV: the parallel-form elements and operators, folded on the CPU       */
/* ------------------------------------------------------------------------ */

/* Filter element a = (F, d, D, eta, J), packed as F[n*n] d[n] D[n*n] eta[n] J[n*n]. */
static int felem_size(int n) { return 3 * n * n + 2 * n; }

/* Eq. (27), literally, with both inverses (I + D_i J_j)^{-1} and (I + J_j D_i)^{-1}. */
int oracle_filter_op(int n, const double *ai, const double *aj, double *out) {
  int nn = n * n, rc = 0;
  const double *Fi = ai, *di = ai + nn, *Di = ai + nn + n, *ei = ai + 2 * nn + n, *Ji = ai + 2 * nn + 2 * n;
  const double *Fj = aj, *dj = aj + nn, *Dj = aj + nn + n, *ej = aj + 2 * nn + n, *Jj = aj + 2 * nn + 2 * n;
  double *Fo = out, *dout = out + nn, *Do = out + nn + n, *eo = out + 2 * nn + n, *Jo = out + 2 * nn + 2 * n;
  double *M1 = dalloc(nn), *M1i = dalloc(nn), *M2 = dalloc(nn), *M2i = dalloc(nn);
  double *FjM1 = dalloc(nn), *FiTM2 = dalloc(nn), *t = dalloc(n), *T = dalloc(nn), *T2 = dalloc(nn);
  eye(n, M1); gemm(n, n, n, 1.0, Di, 0, Jj, 0, 1.0, M1);
  eye(n, M2); gemm(n, n, n, 1.0, Jj, 0, Di, 0, 1.0, M2);
  if (inverse(n, M1, M1i) || inverse(n, M2, M2i)) rc = -1;
  gemm(n, n, n, 1.0, Fj, 0, M1i, 0, 0.0, FjM1);
  gemm(n, n, n, 1.0, Fi, 1, M2i, 0, 0.0, FiTM2);
  /* F_ij */
  gemm(n, n, n, 1.0, FjM1, 0, Fi, 0, 0.0, Fo);
  /* d_ij */
  copy(n, di, t); gemm(n, n, 1, 1.0, Di, 0, ej, 0, 1.0, t);
  gemm(n, n, 1, 1.0, FjM1, 0, t, 0, 0.0, dout); axpy(n, 1.0, dj, dout);
  /* D_ij */
  gemm(n, n, n, 1.0, FjM1, 0, Di, 0, 0.0, T);
  gemm(n, n, n, 1.0, T, 0, Fj, 1, 0.0, Do); axpy(nn, 1.0, Dj, Do);
  /* eta_ij */
  copy(n, ej, t); gemm(n, n, 1, -1.0, Jj, 0, di, 0, 1.0, t);
  gemm(n, n, 1, 1.0, FiTM2, 0, t, 0, 0.0, eo); axpy(n, 1.0, ei, eo);
  /* J_ij */
  gemm(n, n, n, 1.0, FiTM2, 0, Jj, 0, 0.0, T);
  gemm(n, n, n, 1.0, T, 0, Fi, 0, 0.0, T2);
  copy(nn, T2, Jo); axpy(nn, 1.0, Ji, Jo);
  free(M1); free(M1i); free(M2); free(M2i); free(FjM1); free(FiTM2); free(t); free(T); free(T2);
  return rc;
}

/* Smoother element (E, g, S) packed as E[n*n] g[n] S[n*n].  Eq. (30). */
static int selem_size(int n) { return 2 * n * n + n; }
int oracle_smoother_op(int n, const double *ai, const double *aj, double *out) {
  int nn = n * n;
  const double *Ei = ai, *gi = ai + nn, *Si = ai + nn + n;
  const double *Ej = aj, *gj = aj + nn, *Sj = aj + nn + n;
  double *Eo = out, *go = out + nn, *So = out + nn + n, *T = dalloc(nn);
  gemm(n, n, n, 1.0, Ei, 0, Ej, 0, 0.0, Eo);
  gemm(n, n, 1, 1.0, Ei, 0, gj, 0, 0.0, go); axpy(n, 1.0, gi, go);
  gemm(n, n, n, 1.0, Ei, 0, Sj, 0, 0.0, T);
  gemm(n, n, n, 1.0, T, 0, Ei, 1, 0.0, So); axpy(nn, 1.0, Si, So);
  free(T);
  return 0;
}

/* Inclusive scan of N packed elements of size es.  order 0: left-to-right
 * fold; order 1: Hillis-Steele doubling (a different bracketing of the same
 * products).  reverse=0: prefix s_k = a_1 x ... x a_k; reverse=1: suffix
 * s_k = a_k x ... x a_N.  op(n, left, right, out). */
typedef int (*op_t)(int, const double *, const double *, double *);
static int scan(int n, int N, int es, double *a, int order, int reverse, op_t op) {
  int rc = 0;
  double *tmp = dalloc((size_t)es);
  if (order == 0) {
    if (!reverse) {
      for (int k = 1; k < N; ++k) {
        if (op(n, a + (size_t)(k - 1) * es, a + (size_t)k * es, tmp)) rc = -1;
        copy(es, tmp, a + (size_t)k * es);
      }
    } else {
      for (int k = N - 2; k >= 0; --k) {
        if (op(n, a + (size_t)k * es, a + (size_t)(k + 1) * es, tmp)) rc = -1;
        copy(es, tmp, a + (size_t)k * es);
      }
    }
  } else {
    double *b = dalloc((size_t)N * es);
    for (int d = 1; d < N; d *= 2) {
      copy(N * es, a, b);
      for (int k = 0; k < N; ++k) {
        if (!reverse && k >= d) {
          if (op(n, b + (size_t)(k - d) * es, b + (size_t)k * es, a + (size_t)k * es)) rc = -1;
        } else if (reverse && k + d < N) {
          if (op(n, b + (size_t)k * es, b + (size_t)(k + d) * es, a + (size_t)k * es)) rc = -1;
        }
      }
    }
    free(b);
  }
  free(tmp);
  return rc;
}

/* Parallel IMKF (Eq. 25-27) and parallel IMS (Eq. 29-30), folded on the CPU.
 * Outputs (any may be NULL): slow filter x_{k,l}|y_{1:k} (d_k, D_k of the
 * prefix), smoothed first states x_{k,1}|y_{1:N} (g_k, S_k of the suffix).
 * order: 0 sequential fold, 1 doubling bracketing.  flags: ORACLE_LITERAL_SK. */
int oracle_srtm_parallel(int n, int m, int l, int N, const double *A, const double *Q,
                         const double *H, const double *R, const double *m0,
                         const double *P0, const double *y, int order, int flags,
                         double *slow_filt_mean, double *slow_filt_cov,
                         double *first_smooth_mean, double *first_smooth_cov, int nu, const double *B,
                         const double *u) {
  if (n < 1 || m < 1 || l < 1 || N < 1) return -2;
  model_t M;
  model_build(&M, n, m, l, A, Q, H);
  model_inputs(&M, u ? nu : 0, B, H);
  int nn = n * n, fs = felem_size(n), ss = selem_size(n), rc = 0;
  double *bnext = dalloc(n), *yc = dalloc(m), *bl = dalloc(n);
  /* Eq. (25),(26): R_x = M Q~ M^T + R, K = G Q~ M^T R_x^{-1}, F = A_bar - K C_bar,
   * d_k = K y_k, D = Q_bar - K M Q~ G^T, eta_k = C_bar^T R_x^{-1} y_k, J = C_bar^T R_x^{-1} C_bar;
   * with inputs y_k is replaced by y_k - D_bar u_bar_k and d_k gains B_bar u_bar_k (the
   * conditional mean of x_{k,l} given x_{k-1,l} and y_k shifts by the known input terms). */
  double *Rx = dalloc((size_t)m * m), *Rxi = dalloc((size_t)m * m), *K = dalloc((size_t)n * m);
  double *F = dalloc(nn), *D = dalloc(nn), *CtRi = dalloc((size_t)n * m), *J = dalloc(nn);
  copy(m * m, M.MQM, Rx); axpy(m * m, 1.0, R, Rx);
  if (inverse(m, Rx, Rxi)) rc = -1;
  gemm(n, m, m, 1.0, M.GQM, 0, Rxi, 0, 0.0, K);
  copy(nn, M.Abar, F); gemm(n, m, n, -1.0, K, 0, M.Cbar, 0, 1.0, F);
  copy(nn, M.Qbar, D); gemm(n, m, n, -1.0, K, 0, M.GQM, 1, 1.0, D);
  gemm(n, m, m, 1.0, M.Cbar, 1, Rxi, 0, 0.0, CtRi);
  gemm(n, m, n, 1.0, CtRi, 0, M.Cbar, 0, 0.0, J);
  double *fe = dalloc((size_t)N * fs);
  for (int k = 0; k < N; ++k) {
    double *a = fe + (size_t)k * fs;
    const double *yk = y + (size_t)k * m;
    if (k == 0) {   /* F_1 = 0, d_1 = m^f_{1,l}, D_1 = P^f_{1,l}, eta_1 = 0, J_1 = 0 */
      if (imkf_step(&M, R, m0, P0, yk, a + nn, a + nn + n, NULL, UBAR(0))) rc = -1;
    } else {
      copy(m, yk, yc);
      memset(bl, 0, sizeof(double) * n);
      if (M.nu) {
        gemm(m, l * M.nu, 1, -1.0, M.Dbar, 0, UBAR(k), 0, 1.0, yc);
        gemm(n, l * M.nu, 1, 1.0, M.Bbar, 0, UBAR(k), 0, 0.0, bl);
      }
      copy(nn, F, a);
      copy(n, bl, a + nn);
      gemm(n, m, 1, 1.0, K, 0, yc, 0, 1.0, a + nn);
      copy(nn, D, a + nn + n);
      gemm(n, m, 1, 1.0, CtRi, 0, yc, 0, 0.0, a + 2 * nn + n);
      copy(nn, J, a + 2 * nn + 2 * n);
    }
  }
  if (scan(n, N, fs, fe, order, 0, oracle_filter_op)) rc = -1;
  double *mfl = dalloc((size_t)N * n), *Pfl = dalloc((size_t)N * nn);
  for (int k = 0; k < N; ++k) {
    copy(n, fe + (size_t)k * fs + nn, mfl + (size_t)k * n);
    copy(nn, fe + (size_t)k * fs + nn + n, Pfl + (size_t)k * nn);
  }
  if (slow_filt_mean) copy(N * n, mfl, slow_filt_mean);
  if (slow_filt_cov) copy(N * nn, Pfl, slow_filt_cov);

  if (first_smooth_mean || first_smooth_cov) {
    /* Eq. (29): E_k = P^f_{k,1,l} A^T (A P^f_{k,l} A^T + Q)^{-1},
     * g_k = m^f_{k,1} - E_k A m^f_{k,l},  S_k = P^f_{k,1} - E_k A (P^f_{k,1,l})^T;
     * E_N = 0, g_N = m^f_{N,1}, S_N = P^f_{N,1}.  The fast-filter blocks of
     * interval k come from Eq. (17) with the scan's filter result at k-1. */
    double *se = dalloc((size_t)N * ss);
    double *mf = dalloc((size_t)l * n), *Pii = dalloc((size_t)l * nn), *Pil = dalloc((size_t)l * nn);
    double *AP = dalloc(nn), *Pm = dalloc(nn), *PA = dalloc(nn), *Am = dalloc(n), *EA = dalloc(nn);
    for (int k = 0; k < N; ++k) {
      const double *mp = k ? mfl + (size_t)(k - 1) * n : m0;
      const double *Pp = k ? Pfl + (size_t)(k - 1) * nn : P0;
      if (fast_filter_interval(&M, H, R, mp, Pp, y + (size_t)k * m, mf, Pii, Pil, UBAR(k))) rc = -1;
      double *E = se + (size_t)k * ss, *g = E + nn, *S = E + nn + n;
      if (k == N - 1) {
        memset(E, 0, sizeof(double) * nn);
        copy(n, mf, g);
        copy(nn, Pii, S);
        continue;
      }
      gemm(n, n, n, 1.0, A, 0, Pfl + (size_t)k * nn, 0, 0.0, AP);
      gemm(n, n, n, 1.0, AP, 0, A, 1, 0.0, Pm);
      axpy(nn, 1.0, Q, Pm);
      gemm(n, n, n, 1.0, Pil, 0, A, 1, 0.0, PA);                /* P^f_{k,1,l} A^T */
      if (right_solve(n, Pm, n, PA, E)) rc = -1;
      gemm(n, n, 1, 1.0, A, 0, mfl + (size_t)k * n, 0, 0.0, Am);
      if (M.nu) axpy(n, 1.0, BNEXT(k), Am);                      /* + B u_{k,l} */
      copy(n, mf, g); gemm(n, n, 1, -1.0, E, 0, Am, 0, 1.0, g);
      gemm(n, n, n, 1.0, E, 0, A, 0, 0.0, EA);
      copy(nn, Pii, S);
      gemm(n, n, n, -1.0, EA, 0, Pil, (flags & ORACLE_LITERAL_SK) ? 0 : 1, 1.0, S);
    }
    if (scan(n, N, ss, se, order, 1, oracle_smoother_op)) rc = -1;
    for (int k = 0; k < N; ++k) {
      if (first_smooth_mean) copy(n, se + (size_t)k * ss + nn, first_smooth_mean + (size_t)k * n);
      if (first_smooth_cov) copy(nn, se + (size_t)k * ss + nn + n, first_smooth_cov + (size_t)k * nn);
    }
    free(se); free(mf); free(Pii); free(Pil); free(AP); free(Pm); free(PA); free(Am); free(EA);
  }
  free(Rx); free(Rxi); free(K); free(F); free(D); free(CtRi); free(J); free(fe); free(mfl); free(Pfl);
  free(bnext); free(yc); free(bl);
  model_free(&M);
  return rc;
}

/* The lifted slow-rate model of Sec. III-A (Eq. 7-11), for the Riccati pin. */
int oracle_lifted(int n, int m, int l, const double *A, const double *Q, const double *H,
                  double *Abar, double *Qbar, double *Cbar, double *MQM, double *GQM) {
  if (n < 1 || m < 1 || l < 1) return -2;
  model_t M;
  model_build(&M, n, m, l, A, Q, H);
  model_inputs(&M, 0, NULL, H);
  copy(n * n, M.Abar, Abar); copy(n * n, M.Qbar, Qbar); copy(m * n, M.Cbar, Cbar);
  copy(m * m, M.MQM, MQM); copy(n * m, M.GQM, GQM);
  model_free(&M);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* log p(y_{1:N}) by the prediction-error decomposition of the slow-rate     */
/* IMKF (Eq. 9-12): sum_k log N(y_k; C_bar m^f_{k-1,l}, S_k), with           */
/* S_k = C_bar P^f_{k-1,l} C_bar^T + M Q~ M^T + R.  terms (optional, N       */
/* values) receives the per-interval terms.                                  */
/* ------------------------------------------------------------------------ */
int oracle_loglik(int n, int m, int l, int N, const double *A, const double *Q, const double *H,
                  const double *R, const double *m0, const double *P0, const double *y, double *terms,
                  double *total, int nu, const double *B, const double *u) {
  if (n < 1 || m < 1 || l < 1 || N < 1 || !total) return -2;
  model_t M;
  model_build(&M, n, m, l, A, Q, H);
  model_inputs(&M, u ? nu : 0, B, H);
  int rc = 0, nn = n * n;
  double *mf = dalloc((size_t)N * n), *Pf = dalloc((size_t)N * nn), acc = 0.0;
  for (int k = 0; k < N; ++k) {
    const double *mp = k ? mf + (size_t)(k - 1) * n : m0;
    const double *Pp = k ? Pf + (size_t)(k - 1) * nn : P0;
    double t = 0.0;
    if (imkf_step(&M, R, mp, Pp, y + (size_t)k * m, mf + (size_t)k * n, Pf + (size_t)k * nn, &t, UBAR(k))) rc = -1;
    if (terms) terms[k] = t;
    acc += t;
  }
  *total = acc;
  model_free(&M);
  free(mf); free(Pf);
  return rc;
}
