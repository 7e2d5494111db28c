/*
 * CPU oracle for error-vector-sampling deflation / subspace correction ICCG
 * (arXiv 2203.08498). TEST INFRASTRUCTURE ONLY: tests, the package smoke check and the
 * benchmark's CPU-baseline leg call it; the library never does.
 *
 * Plain FP64 C loops written from the paper's definitions, single-threaded as built for the
 * tests. The same source built with OpenMP (the benchmark's all-core timing, in the paper's
 * C/OpenMP style) shares among threads the rows of one colour in the substitutions and the
 * elements of the SpMV and vector loops; the dot products stay serial pairwise sums, so both
 * builds give bit-identical results:
 *   - IC(0) on the pattern of tril(A) (preconditioner M = L L^T, Section 4.4 / 5.3);
 *   - forward / backward substitution taken colour by colour in the given order;
 *   - PCG as in Algorithm "PCG with condition number estimation" (without the power
 *     method), preconditioned by M^{-1} or by the additive subspace correction
 *     M_sc^{-1} = M^{-1} + W (W^T A W)^{-1} W^T (Eq. mc);
 *   - deflated PCG (Algorithm "Deflated PCG") with P = I - W E^{-1} (AW)^T
 *     (Eq. deflation:projector), P^T A p formed explicitly as a vector and the final
 *     correction x = P x_i + W E^{-1} W^T b (Eq. x1);
 *   - sampling method A (Appendix A) or B (Section 4.2, the relative residual levels),
 *     samples taken only while the solve has not stopped;
 *   - the power method of the same algorithm (Section 5.4), run on its own: its vectors
 *     do not depend on the CG iterates, so k steps equal the k products of a k-iteration
 *     solve.
 * Dot products use pairwise summation. E = W^T A W is applied through its dense
 * Cholesky factor. The paper's beta carries a spurious minus sign in Algorithm DPCG; the
 * oracle uses beta = +rho_{i+1}/rho_i, which is the standard CG recurrence.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the parallel loops use: 1 for the serial build. */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

#define ORC_OK 0
#define ORC_ERR_NOT_SPD (-2)
#define ORC_ERR_BREAKDOWN (-3)
#define ORC_ERR_MAXIT (-4)
#define ORC_ERR_STATE (-5)

/* ---------------------------------------------------------------- dot products */

static double pairwise_dot(const double* x, const double* y, long n) {
  if (n <= 32) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
  }
  long h = n / 2;
  return pairwise_dot(x, y, h) + pairwise_dot(x + h, y + h, n - h);
}

double orc_dot(long n, const double* x, const double* y) { return pairwise_dot(x, y, n); }

/* y = A x for CSR A */
void orc_spmv(int n, const int* rp, const int* ci, const double* va, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
    y[i] = s;
  }
}

/* Power method of Algorithm "PCG with condition number estimation" (Section 5.4): v is
 * scaled to unit length, then k times v <- A v, v <- v / ||v||_2 (one step per CG
 * iteration, the product the algorithm forms beside q = A p). Returns the estimate
 * lambda_max = (v, A v) of the final unit vector; v holds that vector. work: n doubles.
 * Returns NaN when a norm is zero or not finite. */
double orc_power_method(int n, const int* rp, const int* ci, const double* va, double* v, int k,
                        double* work) {
  double nv = sqrt(orc_dot(n, v, v));
  if (!(nv > 0.0) || !isfinite(nv)) return NAN;
  for (int i = 0; i < n; ++i) v[i] /= nv;
  for (int step = 0; step < k; ++step) {
    orc_spmv(n, rp, ci, va, v, work);
    nv = sqrt(orc_dot(n, work, work));
    if (!(nv > 0.0) || !isfinite(nv)) return NAN;
    for (int i = 0; i < n; ++i) v[i] = work[i] / nv;
  }
  orc_spmv(n, rp, ci, va, v, work);
  return orc_dot(n, v, work);
}

/* ---------------------------------------------------------------- IC(0) */

/* Number of entries of tril(A) (column <= row). */
long orc_tril_nnz(int n, const int* rp, const int* ci) {
  long c = 0;
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] <= i) ++c;
  return c;
}

/* One IC(0) attempt on A + shift*diag(A), row by row in index order (which is colour order,
 * the rows being colour-major). L has the pattern of tril(A) with the diagonal last in each
 * row. For each row i and each k < i in the pattern:
 *     l_ik = (a_ik - sum_{j<k} l_ij l_kj) / l_kk,
 * the sum running over the common pattern of rows i and k of L; then
 *     l_ii = sqrt(a_ii (1 + shift) - sum_{k<i} l_ik^2).
 * Returns 0, or -(i+1) when the pivot of row i is not positive. */
static long ic0_attempt(int n, const int* rp, const int* ci, const double* va, double shift,
                        const int* Lrp, int* Lci, double* Lva) {
  for (int i = 0; i < n; ++i) {
    int w = Lrp[i];
    double diag = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < i) {
        Lci[w] = ci[k];
        Lva[w] = va[k];
        ++w;
      } else if (ci[k] == i) {
        diag = va[k] * (1.0 + shift);
      }
    }
    Lci[w] = i; /* diagonal last */
    int row_end = w; /* off-diagonal entries of row i are Lrp[i] .. row_end-1 */
    for (int a = Lrp[i]; a < row_end; ++a) {
      int k = Lci[a];
      double s = Lva[a];
      /* merge row i (entries before a, columns < k) with row k (off-diagonals) */
      int pi = Lrp[i], pk = Lrp[k], ek = Lrp[k + 1] - 1;
      while (pi < a && pk < ek) {
        int ji = Lci[pi], jk = Lci[pk];
        if (ji == jk) {
          s -= Lva[pi] * Lva[pk];
          ++pi;
          ++pk;
        } else if (ji < jk) {
          ++pi;
        } else {
          ++pk;
        }
      }
      Lva[a] = s / Lva[Lrp[k + 1] - 1];
    }
    double d = diag;
    for (int a = Lrp[i]; a < row_end; ++a) d -= Lva[a] * Lva[a];
    if (!(d > 0.0)) return -(long)(i + 1);
    Lva[row_end] = sqrt(d);
  }
  return 0;
}

/* IC(0) with the diagonal-shift retry rule: try shift = 0; on a non-positive pivot retry with
 * shift = 1e-3, then double it, up to max_tries attempts. Lrp must hold the row pointer of
 * tril(A) (n+1 entries). Returns 0 and the shift used, or ORC_ERR_NOT_SPD. */
int orc_ic0(int n, const int* rp, const int* ci, const double* va, int max_tries,
            int* Lrp, int* Lci, double* Lva, double* shift_used) {
  Lrp[0] = 0;
  for (int i = 0; i < n; ++i) {
    int c = 0, has_diag = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] <= i) ++c;
      if (ci[k] == i) has_diag = 1;
    }
    if (!has_diag) return ORC_ERR_NOT_SPD; /* IC(0) needs every diagonal entry */
    Lrp[i + 1] = Lrp[i] + c;
  }
  double shift = 0.0;
  for (int t = 0; t < max_tries; ++t) {
    if (ic0_attempt(n, rp, ci, va, shift, Lrp, Lci, Lva) == 0) {
      *shift_used = shift;
      return ORC_OK;
    }
    shift = (shift == 0.0) ? 1e-3 : 2.0 * shift;
  }
  return ORC_ERR_NOT_SPD;
}

/* Transposed index of the strict part of L for the backward sweep: for every row k, the
 * entries a with Lci[a] = k (so Lva[a] = l_jk for the row j owning a), ordered by the colour
 * of j descending and then by j ascending. Urp: n+1 row pointers; Uj[e]: the row j; Ua[e]:
 * the entry a. Returns the number of entries (the strict lower count). */
long orc_ic_transpose(int n, int ncol, const int* cp, const int* Lrp, const int* Lci, int* Urp, int* Uj, int* Ua) {
  for (int k = 0; k <= n; ++k) Urp[k] = 0;
  for (int j = 0; j < n; ++j)
    for (int a = Lrp[j]; a < Lrp[j + 1] - 1; ++a) Urp[Lci[a] + 1] += 1;
  for (int k = 0; k < n; ++k) Urp[k + 1] += Urp[k];
  int* fill = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) fill[k] = Urp[k];
  for (int c = ncol - 1; c >= 0; --c)
    for (int j = cp[c]; j < cp[c + 1]; ++j)
      for (int a = Lrp[j]; a < Lrp[j + 1] - 1; ++a) {
        const int k = Lci[a];
        Uj[fill[k]] = j;
        Ua[fill[k]] = a;
        fill[k] += 1;
      }
  free(fill);
  return Urp[n];
}

/* z = (L L^T)^{-1} r. Forward: for colour c = 0..C-1, every row i of colour c:
 *   y_i = (r_i - sum_{k<i} l_ik y_k) / l_ii.
 * Backward: for colour c = C-1..0, every row i of colour c:
 *   z_i = (y_i - sum_{j>i} l_ji z_j) / l_ii,
 * the sum taken over column i of L (the transposed index of orc_ic_transpose), its terms
 * subtracted one by one from y_i with the later colours first and, within a colour, the rows
 * in ascending order. No two rows of one colour are coupled, so the rows of a colour are
 * independent: with OpenMP they are shared among threads, which changes no result. */
void orc_ic_apply(int n, int ncol, const int* cp, const int* Lrp, const int* Lci, const double* Lva,
                  const int* Urp, const int* Uj, const int* Ua, const double* r, double* z, double* y) {
  (void)n;
  for (int c = 0; c < ncol; ++c) {
#pragma omp parallel for schedule(static)
    for (int i = cp[c]; i < cp[c + 1]; ++i) {
      double s = r[i];
      int e = Lrp[i + 1] - 1;
      for (int a = Lrp[i]; a < e; ++a) s -= Lva[a] * y[Lci[a]];
      y[i] = s / Lva[e];
    }
  }
  for (int c = ncol - 1; c >= 0; --c) {
#pragma omp parallel for schedule(static)
    for (int i = cp[c]; i < cp[c + 1]; ++i) {
      double s = y[i];
      for (int e = Urp[i]; e < Urp[i + 1]; ++e) s -= Lva[Ua[e]] * z[Uj[e]];
      z[i] = s / Lva[Lrp[i + 1] - 1];
    }
  }
}

/* ---------------------------------------------------------------- small dense E */

/* u = E^{-1} f with E = LE LE^T, LE lower triangular, row-major m x m. */
static void chol_solve(int m, const double* LE, const double* f, double* u) {
  for (int i = 0; i < m; ++i) {
    double s = f[i];
    for (int k = 0; k < i; ++k) s -= LE[i * m + k] * u[k];
    u[i] = s / LE[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = u[i];
    for (int k = i + 1; k < m; ++k) s -= LE[k * m + i] * u[k];
    u[i] = s / LE[i * m + i];
  }
}

/* out[k] = sum_i X[i + k n] v[i] for an n x m column-major X */
static void tall_t_vec(long n, int m, const double* X, const double* v, double* out) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < m; ++k) out[k] = pairwise_dot(X + (long)k * n, v, n);
}

/* y += sign * X u */
static void tall_vec_acc(long n, int m, const double* X, const double* u, double sign, double* y) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += X[i + (long)k * n] * u[k];
    y[i] += sign * s;
  }
}

/* ---------------------------------------------------------------- solver */

typedef struct {
  int n;
  const int* rp;
  const int* ci;
  const double* va;
  int ncol;
  const int* cp;
  int precond; /* 0: M = I, 1: IC(0) */
  const int* Lrp;
  const int* Lci;
  const double* Lva;
  const int* Urp; /* transposed index of L (orc_ic_transpose) */
  const int* Uj;
  const int* Ua;
  int mode; /* 0 plain, 1 deflation, 2 subspace correction */
  int m;
  const double* W;  /* n x m column-major */
  const double* AW; /* n x m column-major */
  const double* LE; /* m x m row-major Cholesky factor of E = W^T A W */
} orc_system;

typedef struct {
  double tol;
  int maxit;
  int sample_m;  /* 0: no sampling */
  int lmax;      /* sampling method A parameter, m^lmax > maxit */
  int sample_method; /* 0: method A (Appendix A), 1: method B (residual levels) */
  double* samples;  /* n x sample_m column-major, or NULL */
  int* sample_iter; /* per slot: iteration whose iterate it holds (0 = empty) */
  double* alpha_hist; /* maxit entries or NULL */
  double* beta_hist;  /* maxit entries or NULL */
  double* res_hist;   /* maxit+1 entries of ||r_i||/||b|| or NULL */
  double* wtr_hist;   /* maxit+1 entries of max_k |(W^T r_i)_k| / ||b|| or NULL */
  int iters;
  double relres;
  int status;
} orc_solve_io;

/* Preconditioner: z = M^{-1} r, plus W E^{-1} W^T r in subspace-correction mode (Eq. mc). */
void orc_precond(const orc_system* s, const double* r, double* z, double* work) {
  int n = s->n;
  if (s->precond == 1)
    orc_ic_apply(n, s->ncol, s->cp, s->Lrp, s->Lci, s->Lva, s->Urp, s->Uj, s->Ua, r, z, work);
  else
    memcpy(z, r, sizeof(double) * n);
  if (s->mode == 2 && s->m > 0) {
    double f[64], u[64];
    tall_t_vec(n, s->m, s->W, r, f);
    chol_solve(s->m, s->LE, f, u);
    tall_vec_acc(n, s->m, s->W, u, 1.0, z);
  }
}

/* v = P^T v = v - AW E^{-1} W^T v  (P^T = I - AW E^{-1} W^T, the transpose of Eq.
 * deflation:projector with E symmetric). */
static void apply_PT(const orc_system* s, double* v) {
  double f[64], u[64];
  tall_t_vec(s->n, s->m, s->W, v, f);
  chol_solve(s->m, s->LE, f, u);
  tall_vec_acc(s->n, s->m, s->AW, u, -1.0, v);
}

static double wtr_max(const orc_system* s, const double* r, double bn) {
  if (s->mode != 1 || s->m <= 0) return 0.0;
  double f[64], mx = 0.0;
  tall_t_vec(s->n, s->m, s->W, r, f);
  for (int k = 0; k < s->m; ++k)
    if (fabs(f[k]) > mx) mx = fabs(f[k]);
  return mx / bn;
}

/* Sampling method A (Appendix A) at iteration i (1-based); *h is the algorithm's interval. */
static void sample_a(int i, int m, int lmax, int* h, long n, const double* x, double* samples,
                     int* sample_iter) {
  if (i % *h != 0) return;
  long it = 0, q = i - 1;
  for (int l = 0; l <= lmax; ++l) {
    it += (l % 2 == 0) ? q : -q;
    q /= m;
  }
  int slot = (int)(it % m);
  memcpy(samples + (long)slot * n, x, sizeof(double) * n);
  sample_iter[slot] = i;
  if (i == (*h) * m) *h *= 2;
}

/* Sampling method B (Section 4.2): with the stopping criterion ||r|| <= tol ||b||, the
 * iterate whose relative residual first reaches tol^(s/(m+1)), s = 1..m, is stored. An
 * iteration that first reaches several levels stores its iterate once, in the next slot.
 * The test is made on squares, ||r||^2/||b||^2 <= (tol^2)^(s/(m+1)). reached counts the
 * levels reached so far, used the slots filled. */
static void sample_b(int i, int m, double rel2, double tol2, int* reached, int* used, long n, const double* x,
                     double* samples, int* sample_iter) {
  int lev = *reached;
  while (lev < m && rel2 <= pow(tol2, (double)(lev + 1) / (double)(m + 1))) ++lev;
  if (lev > *reached) {
    memcpy(samples + (long)(*used) * n, x, sizeof(double) * n);
    sample_iter[*used] = i;
    *used += 1;
    *reached = lev;
  }
}

/* Iteration numbers at which sampling method A stores a vector when the solve converges at
 * iteration N (no sample at the converging iteration). slot_iter[m] receives, per slot, the
 * iteration of the vector it finally holds (0 = never filled). */
void orc_sampling_a_schedule(int m, int lmax, int N, int* slot_iter) {
  int h = 1;
  for (int k = 0; k < m; ++k) slot_iter[k] = 0;
  for (int i = 1; i < N; ++i) {
    if (i % h != 0) continue;
    long it = 0, q = i - 1;
    for (int l = 0; l <= lmax; ++l) {
      it += (l % 2 == 0) ? q : -q;
      q /= m;
    }
    slot_iter[(int)(it % m)] = i;
    if (i == h * m) h *= 2;
  }
}

int orc_solve(const orc_system* s, const double* b, double* x, orc_solve_io* io) {
  int n = s->n;
  double* r = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  int status = ORC_OK, h = 1, iters = 0, b_reached = 0, b_used = 0;
  const double bb = orc_dot(n, b, b);
  double bn = sqrt(bb);
  if (io->sample_iter)
    for (int k = 0; k < io->sample_m; ++k) io->sample_iter[k] = 0;
  if (io->sample_m > 0 && s->mode == 1) {
    status = ORC_ERR_STATE; /* sampling is defined on plain / SC iterates only */
    goto done;
  }
  if (bn == 0.0) {
    memset(x, 0, sizeof(double) * n);
    io->relres = 0.0;
    goto done;
  }
  /* r0 = b - A x0 (deflation: r0 = P^T (b - A x0)) */
  orc_spmv(n, s->rp, s->ci, s->va, x, q);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
  if (s->mode == 1) apply_PT(s, r);
  double rn = sqrt(orc_dot(n, r, r));
  if (io->res_hist) io->res_hist[0] = rn / bn;
  if (io->wtr_hist) io->wtr_hist[0] = wtr_max(s, r, bn);
  double rho = 0.0, rho_old = 0.0;
  if (rn > io->tol * bn) {
    for (int i = 1; i <= io->maxit; ++i) {
      orc_precond(s, r, z, w);
      rho = orc_dot(n, r, z);
      if (i == 1) {
        memcpy(p, z, sizeof(double) * n);
      } else {
        double beta = rho / rho_old;
        if (io->beta_hist) io->beta_hist[i - 2] = beta;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n; ++k) p[k] = z[k] + beta * p[k];
      }
      orc_spmv(n, s->rp, s->ci, s->va, p, q);
      if (s->mode == 1) apply_PT(s, q); /* q = P^T A p */
      double pq = orc_dot(n, p, q);
      if (!(pq > 0.0) || !(rho > 0.0)) {
        status = ORC_ERR_BREAKDOWN;
        iters = i - 1;
        break;
      }
      double alpha = rho / pq;
      if (io->alpha_hist) io->alpha_hist[i - 1] = alpha;
#pragma omp parallel for schedule(static)
      for (int k = 0; k < n; ++k) {
        x[k] += alpha * p[k];
        r[k] -= alpha * q[k];
      }
      rho_old = rho;
      iters = i;
      const double rr = orc_dot(n, r, r);
      rn = sqrt(rr);
      if (io->res_hist) io->res_hist[i] = rn / bn;
      if (io->wtr_hist) io->wtr_hist[i] = wtr_max(s, r, bn);
      if (rn <= io->tol * bn) break;
      if (io->sample_m > 0) {
        if (io->sample_method == 1)
          sample_b(i, io->sample_m, rr / bb, io->tol * io->tol, &b_reached, &b_used, n, x, io->samples,
                   io->sample_iter);
        else
          sample_a(i, io->sample_m, io->lmax, &h, n, x, io->samples, io->sample_iter);
      }
      if (i == io->maxit) status = ORC_ERR_MAXIT;
    }
  }
  io->relres = rn / bn;
  if (s->mode == 1) {
    /* x = P x_i + W E^{-1} W^T b = x_i + W E^{-1} (W^T b - (AW)^T x_i) */
    double f1[64], f2[64], u[64];
    tall_t_vec(n, s->m, s->W, b, f1);
    tall_t_vec(n, s->m, s->AW, x, f2);
    for (int k = 0; k < s->m; ++k) f1[k] -= f2[k];
    chol_solve(s->m, s->LE, f1, u);
    tall_vec_acc(n, s->m, s->W, u, 1.0, x);
  }
done:
  io->iters = iters;
  io->status = status;
  free(r);
  free(z);
  free(p);
  free(q);
  free(w);
  return status;
}
