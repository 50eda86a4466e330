/*
 * mlmc_oracle.c -- plain, slow FP64 CPU oracle for the MLMC multigrid hot path.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
 * the benchmark are the only code that may load this library. It shares no source,
 * header or helper with the CUDA library, and neither includes the other.
 *
 * What it computes, following Gmeiner, Drzisga, Ruede, Scheichl, Wohlmuth,
 * "Scheduling massively parallel multigrid for multilevel Monte Carlo methods":
 *   - one sample Y_l = Q_l - Q_{l-1} of the MLMC level difference, both solves on the
 *     same random coefficient sample (Sec. 2.2, Eq. 8 and Algorithm 1);
 *   - the model problem -div(k grad u) = f on D = (0,1)^3 with homogeneous Dirichlet
 *     data (Sec. 3, Eq. 16), with a lognormal coefficient k = exp(Z) (Sec. 3.2);
 *   - the deterministic solve by geometric multigrid (Sec. 7.1 names the cycle family).
 *
 * The concrete discretisation, field model, cycle and quantity of interest are the
 * readings fixed for this library (the paper uses P1 finite elements, an SPDE field
 * sampler and an FMG cycle instead):
 *   grid      nodes x_ijk = (i h, j h, k h), i,j,k in 0..n-1, n = 2^p + 1, h = 1/(n-1);
 *             u = 0 on boundary nodes, unknowns are the interior nodes;
 *   operator  (A u)_p = h^-2 sum_{q in N(p)} k_pq (u_p - u_q), the vertex-centred
 *             7-point finite-volume form with harmonic-mean face coefficients
 *             k_pq = 2 k_p k_q / (k_p + k_q) of the nodal k (boundary nodes included);
 *   field     log k(x) = sigma sqrt(2/M) sum_m cos(w_m . x + b_m), b_m ~ U[0, 2 pi),
 *             drawn by Philox4x32-10, with w_m from the spectral density of the
 *             covariance: Gaussian sigma^2 exp(-r^2 / (2 ell^2)) gives w_m ~ N(0, I/ell^2);
 *             exponential sigma^2 exp(-r / ell) (the paper's covariance, Sec. 3.2) gives
 *             the 3-D multivariate Cauchy law w_m = z / (ell |chi|), z ~ N(0, I),
 *             chi ~ N(0, 1) independent (density proportional to (1 + ell^2 |w|^2)^-2);
 *             or the SPDE sampler of Sec. 3.2 (see the SPDE section below);
 *   cycle     V(nu1, nu2) with red-black Gauss-Seidel, full weighting, trilinear
 *             prolongation, rediscretised coarse operators (k injected), exact dense
 *             Cholesky solve on the 5^3 grid; cycles repeat until ||f-Au||/||f|| <= rtol;
 *   QoI       Q = mean of u over [0.25, 0.75]^3 by the tensor trapezoid rule.
 *
 * Every loop below follows those definitions directly; nothing is blocked, fused or
 * reordered. Compile with -ffp-contract=off so that no multiply-add is contracted. Loops
 * whose nodes are computed independently of each other (field, operator application,
 * residual, one colour of a sweep, restriction, prolongation) run their planes on OpenMP
 * threads when not already inside a parallel region; no node's arithmetic changes, and
 * every sum over nodes stays sequential.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_NOT_CONVERGED (-3)

static const double ORC_PI = 3.14159265358979323846;

/* covariance families of the field */
#define ORC_COV_GAUSS 0
#define ORC_COV_EXP 1
#define ORC_COV_SPDE 2

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 and Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11). One round maps the counter (c0,c1,c2,c3) with
 * key (k0,k1) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
 * the key advances by the Weyl constants (W0, W1) between rounds; ten rounds.
 * The 64-bit variant is kept only so that the round structure can be checked against
 * an independent library implementation of Philox4x64-10.
 * ---------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += W0;
      k[1] += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  /* schoolbook 32x32 partial products, no compiler extensions */
  uint64_t a0 = a & 0xFFFFFFFFu, a1 = a >> 32, b0 = b & 0xFFFFFFFFu, b1 = b >> 32;
  uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  uint64_t mid = (p00 >> 32) + (p01 & 0xFFFFFFFFu) + (p10 & 0xFFFFFFFFu);
  *lo = (mid << 32) | (p00 & 0xFFFFFFFFu);
  *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint64_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += W0;
      k[1] += W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c[0], &hi0, &lo0);
    mulhilo64(M1, c[2], &hi1, &lo1);
    uint64_t n0 = hi1 ^ c[1] ^ k[0];
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c[3] ^ k[1];
    uint64_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* 53-bit uniform in the open interval (0,1) from two 32-bit words. */
static double uniform53(uint32_t a, uint32_t b) {
  double hi = (double)(a >> 5);  /* 27 bits */
  double lo = (double)(b >> 6);  /* 26 bits */
  return (hi * 67108864.0 + lo + 0.5) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------------------
 * Random features of one sample (the realisation omega of one sample of Algorithm 1).
 * Philox key = (run_seed low word, run_seed high word); for feature m and block
 * c = 0,1,2 the counter is (id low word, id high word, m, c). The 12 words give six
 * uniforms U1..U6 from consecutive word pairs; Box-Muller turns (U1,U2) and (U3,U4)
 * into three standard normals g1, g2, g3; w_m = (g1, g2, g3) / ell and b_m = 2 pi U5.
 * ---------------------------------------------------------------------------------- */
void orc_uniforms(uint64_t run_seed, uint64_t sample_id, int m, double U[6]) {
  uint32_t key[2] = {(uint32_t)run_seed, (uint32_t)(run_seed >> 32)};
  uint32_t words[12];
  for (int c = 0; c < 3; ++c) {
    uint32_t ctr[4] = {(uint32_t)sample_id, (uint32_t)(sample_id >> 32), (uint32_t)m, (uint32_t)c};
    orc_philox4x32_10(ctr, key, &words[4 * c]);
  }
  for (int i = 0; i < 6; ++i) U[i] = uniform53(words[2 * i], words[2 * i + 1]);
}

void orc_features(uint64_t run_seed, uint64_t sample_id, int M, double ell, int cov, double* w, double* b) {
  for (int m = 0; m < M; ++m) {
    double U[6];
    orc_uniforms(run_seed, sample_id, m, U);
    double r1 = sqrt(-2.0 * log(U[0]));
    double r2 = sqrt(-2.0 * log(U[2]));
    /* Box-Muller: two independent standard normals from each uniform pair */
    double g1 = r1 * cos(2.0 * ORC_PI * U[1]);
    double g2 = r1 * sin(2.0 * ORC_PI * U[1]);
    double g3 = r2 * cos(2.0 * ORC_PI * U[3]);
    double scale = 1.0 / ell;
    if (cov == ORC_COV_EXP) {
      /* multivariate Cauchy: divide the Gaussian vector by |chi|, chi the fourth normal */
      double chi = r2 * sin(2.0 * ORC_PI * U[3]);
      scale = 1.0 / (ell * fabs(chi));
    }
    w[3 * m + 0] = g1 * scale;
    w[3 * m + 1] = g2 * scale;
    w[3 * m + 2] = g3 * scale;
    b[m] = 2.0 * ORC_PI * U[4];
  }
}

/* log k at one point: sigma sqrt(2/M) sum_m cos(w_m . x + b_m), features in order. */
double orc_logk_point(const double* w, const double* b, int M, double sigma, double x, double y, double z) {
  double s = 0.0;
  for (int m = 0; m < M; ++m) s += cos(w[3 * m] * x + w[3 * m + 1] * y + w[3 * m + 2] * z + b[m]);
  return sigma * sqrt(2.0 / (double)M) * s;
}

/* Nodal coefficient k = exp(log k) at all n^3 nodes (x fastest). */
int orc_field(uint64_t run_seed, uint64_t sample_id, int M, double sigma, double ell, int cov, int n, double* k) {
  if (M <= 0 || n < 2 || (cov != ORC_COV_GAUSS && cov != ORC_COV_EXP)) return ORC_ERR_INVALID;
  double* w = (double*)malloc(sizeof(double) * 3 * (size_t)M);
  double* b = (double*)malloc(sizeof(double) * (size_t)M);
  if (!w || !b) { free(w); free(b); return ORC_ERR_OOM; }
  orc_features(run_seed, sample_id, M, ell, cov, w, b);
  double h = 1.0 / (double)(n - 1);
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
  for (int kz = 0; kz < n; ++kz)
    for (int jy = 0; jy < n; ++jy)
      for (int ix = 0; ix < n; ++ix)
        k[((size_t)kz * n + jy) * n + ix] = exp(orc_logk_point(w, b, M, sigma, ix * h, jy * h, kz * h));
  free(w);
  free(b);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Grid operator. Face coefficients are harmonic means of nodal k. In "mixed" mode the
 * nodal values are first rounded to FP32 and the harmonic mean is evaluated in FP32
 * arithmetic (product, sum, quotient, each rounded); the operator is then applied in
 * FP64 with those FP32-valued faces. That is the operator the FP32-smoother /
 * FP64-refinement solver converges to.
 * ---------------------------------------------------------------------------------- */
static double kface(double a, double b, int mixed) {
  if (mixed) {
    float a32 = (float)a, b32 = (float)b;
    float num = 2.0f * a32 * b32;
    float den = a32 + b32;
    float q = num / den;
    return (double)q;
  }
  return 2.0 * a * b / (a + b);
}

#define IDX(n, i, j, k) (((size_t)(k) * (size_t)(n) + (size_t)(j)) * (size_t)(n) + (size_t)(i))

static int is_interior(int n, int i, int j, int k) {
  return i > 0 && j > 0 && k > 0 && i < n - 1 && j < n - 1 && k < n - 1;
}

/* (A u)_p for an interior node p; boundary u is taken as zero. c >= 0 is the reaction
 * coefficient of -div(k grad u) + c u (0 for the model problem; kappa^2 for the SPDE
 * field sampler of Sec. 3.2). */
static double apply_at(int n, const double* kn, const double* u, int i, int j, int k, int mixed, double c) {
  static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  double h = 1.0 / (double)(n - 1);
  size_t p = IDX(n, i, j, k);
  double up = u[p];
  double s = 0.0;
  for (int d = 0; d < 6; ++d) {
    int qi = i + off[d][0], qj = j + off[d][1], qk = k + off[d][2];
    size_t q = IDX(n, qi, qj, qk);
    double uq = is_interior(n, qi, qj, qk) ? u[q] : 0.0;
    s += kface(kn[p], kn[q], mixed) * (up - uq);
  }
  return s / (h * h) + c * up;
}

/* A u on all interior nodes; boundary entries of Au are set to zero. */
void orc_apply(int n, const double* kn, const double* u, double* Au, int mixed, double c) {
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        Au[IDX(n, i, j, k)] = is_interior(n, i, j, k) ? apply_at(n, kn, u, i, j, k, mixed, c) : 0.0;
}

/* The same operator as a sparse matrix over the interior nodes, numbered x fastest
 * (CSR; at most 7 entries per row, column indices ascending): row p holds
 * -h^-2 k_pq for each interior neighbour q and h^-2 sum_q k_pq + c on the diagonal.
 * indptr has m^3 + 1 entries, indices / data at least 7 m^3 (m = n - 2).
 * Returns the number of stored entries. */
int orc_assemble_csr(int n, const double* kn, int mixed, double c, int* indptr, int* indices, double* data) {
  static const int off[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  int m = n - 2, nnz = 0, row = 0;
  double h = 1.0 / (double)(n - 1);
  for (int k = 1; k < n - 1; ++k)
    for (int j = 1; j < n - 1; ++j)
      for (int i = 1; i < n - 1; ++i) {
        size_t p = IDX(n, i, j, k);
        int prow = (i - 1) + m * ((j - 1) + m * (k - 1));
        double diag = 0.0;
        indptr[row++] = nnz;
        int diag_pos = -1;
        for (int d = 0; d < 6; ++d) {
          int qi = i + off[d][0], qj = j + off[d][1], qk = k + off[d][2];
          double kf = kface(kn[p], kn[IDX(n, qi, qj, qk)], mixed);
          diag += kf;
          if (d == 3 && diag_pos < 0) { diag_pos = nnz; indices[nnz] = prow; data[nnz] = 0.0; ++nnz; }
          if (is_interior(n, qi, qj, qk)) {
            indices[nnz] = (qi - 1) + m * ((qj - 1) + m * (qk - 1));
            data[nnz] = -kf / (h * h);
            ++nnz;
          }
        }
        data[diag_pos] = diag / (h * h) + c;
      }
  indptr[row] = nnz;
  return nnz;
}

/* r = f - A u on interior nodes, zero on the boundary. f == NULL means f = 1. */
void orc_residual(int n, const double* kn, const double* f, const double* u, double* r, int mixed, double c) {
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        size_t p = IDX(n, i, j, k);
        if (!is_interior(n, i, j, k)) { r[p] = 0.0; continue; }
        double fp = f ? f[p] : 1.0;
        r[p] = fp - apply_at(n, kn, u, i, j, k, mixed, c);
      }
}

/* One red-black Gauss-Seidel sweep: red nodes ((i+j+k) even) first, then black.
 * u_p <- (h^2 f_p + sum_q k_pq u_q) / (sum_q k_pq + c h^2) with boundary u_q = 0. */
void orc_rbgs_sweep(int n, const double* kn, const double* f, double* u, int mixed, double c) {
  static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  double h = 1.0 / (double)(n - 1);
  for (int colour = 0; colour < 2; ++colour) {
    /* a node of one colour reads only nodes of the other: any order gives the same values */
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
    for (int k = 1; k < n - 1; ++k)
      for (int j = 1; j < n - 1; ++j)
        for (int i = 1; i < n - 1; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          size_t p = IDX(n, i, j, k);
          double num = h * h * (f ? f[p] : 1.0), den = 0.0;
          for (int d = 0; d < 6; ++d) {
            int qi = i + off[d][0], qj = j + off[d][1], qk = k + off[d][2];
            size_t q = IDX(n, qi, qj, qk);
            double kf = kface(kn[p], kn[q], mixed);
            num += kf * (is_interior(n, qi, qj, qk) ? u[q] : 0.0);
            den += kf;
          }
          u[p] = num / (den + c * h * h);
        }
  }
}

/* Full weighting: coarse value at interior coarse node I is
 * sum over offsets d in {-1,0,1}^3 of (1/64) prod_a (2 - |d_a|) * r(2I + d).
 * Coarse boundary values are zero. */
void orc_restrict_fw(int nf, const double* r, double* rc) {
  int nc = (nf + 1) / 2;
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
  for (int K = 0; K < nc; ++K)
    for (int J = 0; J < nc; ++J)
      for (int I = 0; I < nc; ++I) {
        size_t P = IDX(nc, I, J, K);
        if (!is_interior(nc, I, J, K)) { rc[P] = 0.0; continue; }
        double s = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              double wgt = (double)((2 - abs(dx)) * (2 - abs(dy)) * (2 - abs(dz))) / 64.0;
              s += wgt * r[IDX(nf, 2 * I + dx, 2 * J + dy, 2 * K + dz)];
            }
        rc[P] = s;
      }
}

/* Trilinear interpolation of the coarse correction, added on interior fine nodes:
 * the fine node (i,j,k) lies between coarse nodes floor(i/2)..ceil(i/2) per axis,
 * with weight 1 on a coincident axis and 1/2 on each neighbour otherwise. */
void orc_prolong_add(int nf, const double* ec, double* u) {
  int nc = (nf + 1) / 2;
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
  for (int k = 1; k < nf - 1; ++k)
    for (int j = 1; j < nf - 1; ++j)
      for (int i = 1; i < nf - 1; ++i) {
        int ia[2] = {i / 2, (i + 1) / 2}, ja[2] = {j / 2, (j + 1) / 2}, ka[2] = {k / 2, (k + 1) / 2};
        double s = 0.0;
        for (int c = 0; c < 8; ++c) {
          int I = ia[c & 1], J = ja[(c >> 1) & 1], K = ka[(c >> 2) & 1];
          s += 0.125 * ec[IDX(nc, I, J, K)];
        }
        u[IDX(nf, i, j, k)] += s;
      }
}

/* ------------------------------------------------------------------------------------
 * Exact coarsest-grid solve: assemble the dense matrix of A on the interior nodes
 * (column by column, by applying A to unit vectors), factor A = L L^T by Cholesky,
 * and solve by forward and backward substitution.
 * ---------------------------------------------------------------------------------- */
int orc_coarse_solve(int n, const double* kn, const double* f, double* u, int mixed, double c) {
  int m = n - 2, N = m * m * m;
  size_t n3 = (size_t)n * n * n;
  double* A = (double*)calloc((size_t)N * N, sizeof(double));
  double* e = (double*)calloc(n3, sizeof(double));
  double* Ae = (double*)calloc(n3, sizeof(double));
  double* y = (double*)calloc((size_t)N, sizeof(double));
  int status = ORC_OK;
  if (!A || !e || !Ae || !y) { status = ORC_ERR_OOM; goto done; }
  for (int col = 0; col < N; ++col) {
    int ci = 1 + col % m, cj = 1 + (col / m) % m, ck = 1 + col / (m * m);
    memset(e, 0, n3 * sizeof(double));
    e[IDX(n, ci, cj, ck)] = 1.0;
    orc_apply(n, kn, e, Ae, mixed, c);
    for (int r = 0; r < N; ++r) {
      int ri = 1 + r % m, rj = 1 + (r / m) % m, rk = 1 + r / (m * m);
      A[(size_t)r * N + col] = Ae[IDX(n, ri, rj, rk)];
    }
  }
  /* Cholesky, lower triangle in place */
  for (int j = 0; j < N; ++j) {
    double d = A[(size_t)j * N + j];
    for (int p = 0; p < j; ++p) d -= A[(size_t)j * N + p] * A[(size_t)j * N + p];
    if (!(d > 0.0)) { status = ORC_ERR_INVALID; goto done; }
    double ljj = sqrt(d);
    A[(size_t)j * N + j] = ljj;
    for (int i = j + 1; i < N; ++i) {
      double s = A[(size_t)i * N + j];
      for (int p = 0; p < j; ++p) s -= A[(size_t)i * N + p] * A[(size_t)j * N + p];
      A[(size_t)i * N + j] = s / ljj;
    }
  }
  /* L y = f */
  for (int i = 0; i < N; ++i) {
    int ii = 1 + i % m, ij = 1 + (i / m) % m, ik = 1 + i / (m * m);
    double s = f ? f[IDX(n, ii, ij, ik)] : 1.0;
    for (int p = 0; p < i; ++p) s -= A[(size_t)i * N + p] * y[p];
    y[i] = s / A[(size_t)i * N + i];
  }
  /* L^T x = y, written into the interior of u */
  for (int i = N - 1; i >= 0; --i) {
    double s = y[i];
    for (int p = i + 1; p < N; ++p) s -= A[(size_t)p * N + i] * y[p];
    y[i] = s / A[(size_t)i * N + i];
  }
  memset(u, 0, n3 * sizeof(double));
  for (int i = 0; i < N; ++i) {
    int ii = 1 + i % m, ij = 1 + (i / m) % m, ik = 1 + i / (m * m);
    u[IDX(n, ii, ij, ik)] = y[i];
  }
done:
  free(A); free(e); free(Ae); free(y);
  return status;
}

/* ------------------------------------------------------------------------------------
 * Multigrid hierarchy and V-cycle.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int levels;      /* number of grids, finest first */
  int n[32];
  double* k[32];   /* nodal coefficient per grid: injection of the finest k */
  double* f[32];   /* right-hand side per grid (grid 0: the caller's f or NULL) */
  double* u[32];   /* iterate / correction per grid */
  double* r[32];   /* residual scratch per grid */
} orc_hierarchy;

static void hier_free(orc_hierarchy* H) {
  for (int l = 0; l < H->levels; ++l) {
    if (l > 0) { free(H->k[l]); free(H->f[l]); free(H->u[l]); }
    free(H->r[l]);
  }
}

/* Injection: coarse node I is fine node 2I. */
static void inject(int nf, const double* kf, double* kc) {
  int nc = (nf + 1) / 2;
  for (int K = 0; K < nc; ++K)
    for (int J = 0; J < nc; ++J)
      for (int I = 0; I < nc; ++I) kc[IDX(nc, I, J, K)] = kf[IDX(nf, 2 * I, 2 * J, 2 * K)];
}

static int valid_n(int n) {
  if (n < 5) return 0;
  int m = n - 1;
  return (m & (m - 1)) == 0;
}

static int hier_build(orc_hierarchy* H, int n, const double* k, const double* f, double* u) {
  memset(H, 0, sizeof(*H));
  int nl = n, l = 0;
  while (1) {
    H->n[l] = nl;
    if (nl == 5) break;
    nl = (nl + 1) / 2;
    ++l;
  }
  H->levels = l + 1;
  H->k[0] = (double*)k;
  H->f[0] = (double*)f;
  H->u[0] = u;
  for (l = 0; l < H->levels; ++l) {
    size_t n3 = (size_t)H->n[l] * H->n[l] * H->n[l];
    if (l > 0) {
      H->k[l] = (double*)malloc(n3 * sizeof(double));
      H->f[l] = (double*)calloc(n3, sizeof(double));
      H->u[l] = (double*)calloc(n3, sizeof(double));
      if (!H->k[l] || !H->f[l] || !H->u[l]) { H->levels = l + 1; return ORC_ERR_OOM; }
      inject(H->n[l - 1], H->k[l - 1], H->k[l]);
    }
    H->r[l] = (double*)calloc(n3, sizeof(double));
    if (!H->r[l]) { H->levels = l + 1; return ORC_ERR_OOM; }
  }
  return ORC_OK;
}

/* One V(nu1, nu2) cycle on grid l of the hierarchy (u[l] is updated in place). */
static int vcycle(orc_hierarchy* H, int l, int nu1, int nu2, int mixed, double c) {
  int n = H->n[l];
  if (l == H->levels - 1) return orc_coarse_solve(n, H->k[l], H->f[l], H->u[l], mixed, c);
  for (int s = 0; s < nu1; ++s) orc_rbgs_sweep(n, H->k[l], H->f[l], H->u[l], mixed, c);
  orc_residual(n, H->k[l], H->f[l], H->u[l], H->r[l], mixed, c);
  orc_restrict_fw(n, H->r[l], H->f[l + 1]);
  size_t nc3 = (size_t)H->n[l + 1] * H->n[l + 1] * H->n[l + 1];
  memset(H->u[l + 1], 0, nc3 * sizeof(double));
  int st = vcycle(H, l + 1, nu1, nu2, mixed, c);
  if (st != ORC_OK) return st;
  orc_prolong_add(n, H->u[l + 1], H->u[l]);
  for (int s = 0; s < nu2; ++s) orc_rbgs_sweep(n, H->k[l], H->f[l], H->u[l], mixed, c);
  return ORC_OK;
}

/* Discrete l2 norm over interior nodes. */
static double interior_norm(int n, const double* v) {
  double s = 0.0;
  for (int k = 1; k < n - 1; ++k)
    for (int j = 1; j < n - 1; ++j)
      for (int i = 1; i < n - 1; ++i) s += v[IDX(n, i, j, k)] * v[IDX(n, i, j, k)];
  return sqrt(s);
}

/*
 * Solve A u = f by V(nu1, nu2) cycles from the caller's initial guess in u (boundary
 * entries are forced to zero). After each cycle the relative residual
 * ||f - A u||_2 / ||f||_2 over interior nodes is recorded in res_hist[c] (if not
 * NULL); cycling stops when it is <= rtol or after max_cycles cycles, which returns
 * ORC_ERR_NOT_CONVERGED (u still holds the last iterate). rtol <= 0 runs exactly
 * max_cycles cycles and returns ORC_OK.
 */
int orc_mg_solve(int n, const double* k, const double* f, double* u, int nu1, int nu2, double rtol,
                 int max_cycles, int mixed, double c, int* cycles_out, double* relres_out, double* res_hist) {
  if (!valid_n(n) || nu1 < 0 || nu2 < 0 || max_cycles < 0 || !(c >= 0.0)) return ORC_ERR_INVALID;
  size_t n3 = (size_t)n * n * n;
  for (int kz = 0; kz < n; ++kz)
    for (int jy = 0; jy < n; ++jy)
      for (int ix = 0; ix < n; ++ix)
        if (!is_interior(n, ix, jy, kz)) u[IDX(n, ix, jy, kz)] = 0.0;
  orc_hierarchy H;
  int st = hier_build(&H, n, k, f, u);
  if (st != ORC_OK) { hier_free(&H); return st; }
  double* fone = NULL;
  if (!f) {
    fone = (double*)malloc(n3 * sizeof(double));
    if (!fone) { hier_free(&H); return ORC_ERR_OOM; }
    for (size_t p = 0; p < n3; ++p) fone[p] = 1.0;
  }
  const double* fe = f ? f : fone;
  double fnorm = interior_norm(n, fe);
  double relres = 0.0;
  orc_residual(n, k, f, u, H.r[0], mixed, c);
  relres = interior_norm(n, H.r[0]) / fnorm;
  int cyc = 0;
  int status = ORC_OK;
  if (rtol > 0.0 && relres <= rtol) goto finish;
  for (cyc = 0; cyc < max_cycles;) {
    st = vcycle(&H, 0, nu1, nu2, mixed, c);
    if (st != ORC_OK) { status = st; goto finish; }
    ++cyc;
    orc_residual(n, k, f, u, H.r[0], mixed, c);
    relres = interior_norm(n, H.r[0]) / fnorm;
    if (res_hist) res_hist[cyc - 1] = relres;
    if (rtol > 0.0 && relres <= rtol) break;
  }
  if (rtol > 0.0 && relres > rtol) status = ORC_ERR_NOT_CONVERGED;
finish:
  if (cycles_out) *cycles_out = cyc;
  if (relres_out) *relres_out = relres;
  free(fone);
  hier_free(&H);
  return status;
}

/* Q = mean of u over [0.25,0.75]^3 = 8 * h^3 * sum_S w_i w_j w_k u_ijk, with S the
 * nodes (n-1)/4 .. 3(n-1)/4 per axis and trapezoid weights 1/2 at both ends. */
double orc_qoi(int n, const double* u) {
  int lo = (n - 1) / 4, hi = 3 * (n - 1) / 4;
  double h = 1.0 / (double)(n - 1);
  double s = 0.0;
  for (int k = lo; k <= hi; ++k)
    for (int j = lo; j <= hi; ++j)
      for (int i = lo; i <= hi; ++i) {
        double wi = (i == lo || i == hi) ? 0.5 : 1.0;
        double wj = (j == lo || j == hi) ? 0.5 : 1.0;
        double wk = (k == lo || k == hi) ? 0.5 : 1.0;
        s += wi * wj * wk * u[IDX(n, i, j, k)];
      }
  return 8.0 * h * h * h * s;
}

/* ------------------------------------------------------------------------------------
 * SPDE field sampler (Sec. 3.2): Z solves (kappa^2 - Laplace) Z = W, W Gaussian white
 * noise, on a box around D with homogeneous Neumann data. In R^3 the solution has the
 * covariance (8 pi kappa)^-1 exp(-kappa r) (the Green's function exp(-kappa r)/(4 pi r)
 * convolved with itself; Whittle), so kappa = 1 / lambda gives the exponential
 * covariance of the paper's field with correlation length lambda = ell, and
 * log k = sqrt(8 pi kappa sigma^2) Z has variance sigma^2 and covariance
 * sigma^2 exp(-r / lambda). (The paper's lambda = 2 / kappa is the "practical range"
 * sqrt(8 nu) / kappa at nu = 1/2, at odds with its own covariance formula; this file
 * follows the covariance formula.)
 *
 * Discretisation (readings of this library; the paper uses P1 finite elements):
 *   - cell-centred finite volumes on a box around D: for the level grid n of D (spacing
 *     h = 1/(n-1)) the box (-1/2 - h/2, 3/2 - h/2)^3 of C = 2(n-1) cells of side h per
 *     axis, cell i centred at -1/2 + i h, so D's node j is the centre of cell
 *     j + (n-1)/2 (margin 1/2 around D; the paper's box is (-1, 2)^3);
 *   - cell p, scaled by 1/h: (kappa^2 h^2 + n_p) Z_p - sum_q Z_q = W(cell p) / h, the
 *     sum over the n_p face neighbours inside the box (zero flux through the box);
 *   - W(cell) is exact white noise integrated over the cell: the cells of the pair's
 *     fine grid n_f (spacing h_f) and of its coarse grid (2 h_f) are unions of octants,
 *     cubes of side h_f/2 tiling (-1/2 - h_f, 3/2 - h_f/2)^3 (4(n_f - 1) + 1 per axis),
 *     each carrying (h_f/2)^(3/2) xi with one standard normal xi per octant, so both
 *     grids of one sample see the same realisation of W.
 *
 * The normals: Marsaglia's polar method (Marsaglia and Bray 1964) on Philox4x32-10
 * words, in FP32 with only correctly rounded operations (+, *, /, sqrt, fma) and the
 * natural logarithm below, so that any IEEE implementation reproduces them exactly.
 * ---------------------------------------------------------------------------------- */

/* ln s for normal s > 0 in FP32: s = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m =
 * 2 atanh(t) = 2 t (1 + t^2/3 + t^4/5 + ... + t^10/11), t = (m - 1)/(m + 1), |t| < 0.172
 * (the series of ln((1+t)/(1-t))), and e ln 2 with ln 2 split into a 16-bit head and a
 * tail (Cody and Waite), every step rounded once. */
float orc_log_series(float s) {
  uint32_t b;
  memcpy(&b, &s, sizeof b);
  int e = (int)((b >> 23) & 0xffu) - 127;
  uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mb, sizeof m);
  if (m > 0x1.6a09e6p+0f) {
    m = 0.5f * m;
    e += 1;
  }
  float t = (m - 1.0f) / (m + 1.0f);
  float t2 = t * t;
  float p = fmaf(t2, 0x1.745d18p-4f, 0x1.c71c72p-4f);
  p = fmaf(t2, p, 0x1.24924ap-3f);
  p = fmaf(t2, p, 0x1.99999ap-3f);
  p = fmaf(t2, p, 0x1.555556p-2f);
  p = fmaf(t2, p, 1.0f);
  float lm = (2.0f * t) * p;
  float fe = (float)e;
  return fmaf(fe, 0x1.62e400p-1f, fmaf(fe, 0x1.7f7d1cp-20f, lm));
}

/* Standard normal of octant `oct` of sample `sample_id`: attempt a = 0..31 takes the
 * word pair (2(a&1), 2(a&1)+1) of Philox4x32-10 with key (seed lo, seed hi) and counter
 * (id lo, id hi, oct lo, 0x5D000000 | (a>>1) << 8 | oct >> 32); a word w gives
 * U = ((w >> 8) - 2^23 + 1/2) 2^-23 in (-1, 1); the first pair with 0 < s = U1^2 + U2^2
 * < 1 returns U1 sqrt(-2 ln s / s); none in 32 attempts (probability 5e-22) returns 0. */
float orc_octant_normal(uint64_t run_seed, uint64_t sample_id, uint64_t oct) {
  uint32_t key[2] = {(uint32_t)run_seed, (uint32_t)(run_seed >> 32)};
  for (int call = 0; call < 16; ++call) {
    uint32_t ctr[4] = {(uint32_t)sample_id, (uint32_t)(sample_id >> 32), (uint32_t)oct,
                       0x5D000000u | ((uint32_t)call << 8) | (uint32_t)(oct >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int half = 0; half < 2; ++half) {
      float u1 = ((float)((int32_t)(w[2 * half] >> 8) - 8388608) + 0.5f) * 0x1p-23f;
      float u2 = ((float)((int32_t)(w[2 * half + 1] >> 8) - 8388608) + 0.5f) * 0x1p-23f;
      float t = u2 * u2;
      float sq = fmaf(u1, u1, t);
      if (sq > 0.0f && sq < 1.0f) {
        float q = (-2.0f * orc_log_series(sq)) / sq;
        return u1 * sqrtf(q);
      }
    }
  }
  return 0.0f;
}

static int spde_sizes_ok(int n, int n_noise) {
  return valid_n(n) && (n_noise == n || n_noise == 2 * n - 1) && n_noise <= 1025;
}

/* Scaled right-hand side g_p = W(cell p) / h on the C^3 cells (C = 2(n-1), x fastest)
 * of level grid n for the pair whose fine grid is n_noise (n, or 2n - 1 for the coarse
 * grid of a pair): the octants of cell i along an axis are 2 r i + 2 - r .. 2 r i + 1 + r
 * with r = h / h_f in {1, 2}; sums taken z, y, x outermost to
 * innermost. */
int orc_spde_noise(uint64_t run_seed, uint64_t sample_id, int n, int n_noise, double* g) {
  if (!spde_sizes_ok(n, n_noise)) return ORC_ERR_INVALID;
  int C = 2 * (n - 1);
  long r = (long)((n_noise - 1) / (n - 1));
  uint64_t Mo = 4 * (uint64_t)(n_noise - 1) + 1;
  double h = 1.0 / (double)(n - 1), hf = 1.0 / (double)(n_noise - 1);
  double v = 0.5 * hf;
  double scale = sqrt(v * v * v) / h;
  for (long K = 0; K < C; ++K)
    for (long J = 0; J < C; ++J)
      for (long I = 0; I < C; ++I) {
        long az0 = 2 * r * K + 2 - r, ay0 = 2 * r * J + 2 - r, ax0 = 2 * r * I + 2 - r;
        double sum = 0.0;
        for (long az = az0; az < az0 + 2 * r; ++az)
          for (long ay = ay0; ay < ay0 + 2 * r; ++ay)
            for (long ax = ax0; ax < ax0 + 2 * r; ++ax)
              sum += (double)orc_octant_normal(run_seed, sample_id,
                                               ((uint64_t)az * Mo + (uint64_t)ay) * Mo + (uint64_t)ax);
        g[((size_t)K * C + (size_t)J) * C + (size_t)I] = scale * sum;
      }
  return ORC_OK;
}

/* The scaled SPDE operator on the C^3 cells: (A Z)_p = (c h^2 + n_p) Z_p - sum_q Z_q. */
void orc_spde_apply(int C, double ch2, const double* Z, double* AZ) {
  for (int k = 0; k < C; ++k)
    for (int j = 0; j < C; ++j)
      for (int i = 0; i < C; ++i) {
        size_t p = ((size_t)k * C + j) * C + i;
        double s = 0.0;
        int np = 0;
        if (i > 0) { s += Z[p - 1]; ++np; }
        if (i < C - 1) { s += Z[p + 1]; ++np; }
        if (j > 0) { s += Z[p - C]; ++np; }
        if (j < C - 1) { s += Z[p + C]; ++np; }
        if (k > 0) { s += Z[p - (size_t)C * C]; ++np; }
        if (k < C - 1) { s += Z[p + (size_t)C * C]; ++np; }
        AZ[p] = (ch2 + (double)np) * Z[p] - s;
      }
}

/* Transform along one axis of a C^3 array: out[.., a, ..] = sum_b M[a][b] in[.., b, ..],
 * axis 0 = x (stride 1), 1 = y (stride C), 2 = z (stride C^2). */
static void axis_transform(int C, const double* M, const double* in, double* out, int axis) {
  size_t st = axis == 0 ? 1 : (axis == 1 ? (size_t)C : (size_t)C * C);
  for (int k = 0; k < C; ++k)
    for (int j = 0; j < C; ++j)
      for (int i = 0; i < C; ++i) {
        int idx[3] = {i, j, k};
        size_t p = ((size_t)k * C + j) * C + i;
        size_t base = p - (size_t)idx[axis] * st;
        double s = 0.0;
        for (int b = 0; b < C; ++b) s += M[(size_t)idx[axis] * C + b] * in[base + (size_t)b * st];
        out[p] = s;
      }
}

/* Exact solve of A Z = g by the eigenvectors of the one-dimensional zero-flux
 * second-difference matrix (the orthonormal DCT-II basis phi_a(i) = w_a cos(pi a (i +
 * 1/2) / C), eigenvalue 4 sin^2(pi a / (2 C))): transform along the three axes, divide
 * by c h^2 + the three eigenvalues, transform back. */
int orc_spde_solve(int C, double ch2, const double* g, double* Z) {
  if (C < 1 || !(ch2 > 0.0)) return ORC_ERR_INVALID;
  size_t C3 = (size_t)C * C * C;
  double* P = (double*)malloc((size_t)C * C * sizeof(double));   /* P[a][i] = phi_a(i) */
  double* Pt = (double*)malloc((size_t)C * C * sizeof(double));  /* transpose */
  double* lam = (double*)malloc((size_t)C * sizeof(double));
  double* t1 = (double*)malloc(C3 * sizeof(double));
  double* t2 = (double*)malloc(C3 * sizeof(double));
  int st = ORC_OK;
  if (!P || !Pt || !lam || !t1 || !t2) { st = ORC_ERR_OOM; goto done; }
  for (int a = 0; a < C; ++a) {
    double w = a == 0 ? sqrt(1.0 / C) : sqrt(2.0 / C);
    double sn = sin(ORC_PI * a / (2.0 * C));
    lam[a] = 4.0 * sn * sn;
    for (int i = 0; i < C; ++i) {
      P[(size_t)a * C + i] = w * cos(ORC_PI * a * (i + 0.5) / C);
      Pt[(size_t)i * C + a] = P[(size_t)a * C + i];
    }
  }
  axis_transform(C, P, g, t1, 0);
  axis_transform(C, P, t1, t2, 1);
  axis_transform(C, P, t2, t1, 2);
  for (int k = 0; k < C; ++k)
    for (int j = 0; j < C; ++j)
      for (int i = 0; i < C; ++i) t1[((size_t)k * C + j) * C + i] /= ch2 + lam[i] + lam[j] + lam[k];
  axis_transform(C, Pt, t1, t2, 0);
  axis_transform(C, Pt, t2, t1, 1);
  axis_transform(C, Pt, t1, Z, 2);
done:
  free(P); free(Pt); free(lam); free(t1); free(t2);
  return st;
}

/* k = exp(log k) at the n^3 nodes of D for the SPDE field: the noise of orc_spde_noise,
 * the exact solve with kappa = 1 / lambda, log k = sqrt(8 pi kappa sigma2) Z at the
 * cells centred on D's nodes. */
int orc_spde_field(uint64_t run_seed, uint64_t sample_id, double sigma2, double lambda, int n, int n_noise,
                   double* k) {
  if (!spde_sizes_ok(n, n_noise) || !(lambda > 0.0) || !(sigma2 >= 0.0)) return ORC_ERR_INVALID;
  int C = 2 * (n - 1), off = (n - 1) / 2;
  size_t C3 = (size_t)C * C * C;
  double* g = (double*)malloc(C3 * sizeof(double));
  double* Z = (double*)malloc(C3 * sizeof(double));
  int st = ORC_OK;
  if (!g || !Z) { st = ORC_ERR_OOM; goto done; }
  st = orc_spde_noise(run_seed, sample_id, n, n_noise, g);
  if (st != ORC_OK) goto done;
  {
    double h = 1.0 / (double)(n - 1), kappa = 1.0 / lambda;
    st = orc_spde_solve(C, kappa * kappa * h * h, g, Z);
    if (st != ORC_OK) goto done;
    double a = sqrt(8.0 * ORC_PI * kappa * sigma2);
    for (int kz = 0; kz < n; ++kz)
      for (int jy = 0; jy < n; ++jy)
        for (int ix = 0; ix < n; ++ix)
          k[IDX(n, ix, jy, kz)] = exp(a * Z[((size_t)(kz + off) * C + (size_t)(jy + off)) * C + (size_t)(ix + off)]);
  }
done:
  free(g);
  free(Z);
  return st;
}

/* ------------------------------------------------------------------------------------
 * One MLMC sample (Algorithm 1): set up the coefficient of the
 * realisation `sample_id` on the fine grid n_fine and (if n_coarse > 0) on the
 * coarse grid n_coarse, solve both with f = 1, and return Q on each grid.
 * Each grid evaluates the field at its own nodes.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  uint64_t run_seed;
  double sigma2;
  double ell;
  int M;
  int nu1, nu2;
  double rtol;
  int max_cycles;
  int mixed;
  int cov; /* ORC_COV_GAUSS, ORC_COV_EXP or ORC_COV_SPDE */
} orc_cfg;

/* n_noise: the grid of the pair's fine solve (the SPDE white noise lives on its octants). */
static int solve_q(const orc_cfg* c, uint64_t sample_id, int n, int n_noise, double* Q, int* cycles) {
  size_t n3 = (size_t)n * n * n;
  double* k = (double*)malloc(n3 * sizeof(double));
  double* u = (double*)calloc(n3, sizeof(double));
  if (!k || !u) { free(k); free(u); return ORC_ERR_OOM; }
  int st;
  if (c->cov == ORC_COV_SPDE)
    st = orc_spde_field(c->run_seed, sample_id, c->sigma2, c->ell, n, n_noise, k);
  else
    st = orc_field(c->run_seed, sample_id, c->M, sqrt(c->sigma2), c->ell, c->cov, n, k);
  if (st == ORC_OK) {
    double relres;
    st = orc_mg_solve(n, k, NULL, u, c->nu1, c->nu2, c->rtol, c->max_cycles, c->mixed, 0.0, cycles, &relres, NULL);
    *Q = orc_qoi(n, u);
  }
  free(k);
  free(u);
  return st;
}

int orc_sample(const orc_cfg* c, int n_fine, int n_coarse, uint64_t sample_id, double* Qf, double* Qc,
               int* cycles_f, int* cycles_c) {
  int st = solve_q(c, sample_id, n_fine, n_fine, Qf, cycles_f);
  if (st != ORC_OK) return st;
  *Qc = 0.0;
  *cycles_c = 0;
  if (n_coarse > 0) st = solve_q(c, sample_id, n_coarse, n_fine, Qc, cycles_c);
  return st;
}

/* A batch of independent samples, OpenMP over samples only (no other parallelism).
 * Y[i] = Qf[i] - Qc[i] (Qc = 0 for level 0). Returns the first non-OK status. */
int orc_level_batch(const orc_cfg* c, int n_fine, int n_coarse, const uint64_t* ids, int N, double* Y,
                    double* Qf, double* Qc, int* cycles_f, int* cycles_c, int nthreads) {
  int status = ORC_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < N; ++i) {
    int st = orc_sample(c, n_fine, n_coarse, ids[i], &Qf[i], &Qc[i], &cycles_f[i], &cycles_c[i]);
    Y[i] = Qf[i] - Qc[i];
    if (st != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
      if (status == ORC_OK) status = st;
    }
  }
  return status;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
