/*
 * dh_oracle.c -- TEST INFRASTRUCTURE. A plain, slow FP64 CPU oracle for the
 * data-parallel path of "Real-time digital holography of the retina by principal
 * component analysis" (Puyo et al., arXiv 2004.00923).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's shared library. It shares no code, header, table or helper with the
 * CUDA library: it has its own radix-2 FFT, chirp, covariance, Jacobi
 * eigensolver and projection, each written straight from the paper's equations.
 *
 * Notation (the paper's): a window is n_t frames I(x, y, t) of n_x x n_y pixels.
 *   Eq. 1  Fresnel transform, evaluated with one spatial FFT per frame.
 *   Eq. 4  C = H^{t*} H, H the (n_x n_y, n_t) space-time matrix of holograms.
 *   Eq. 5  C = V Lambda V^{t*}  (Hermitian eigendecomposition).
 *   Eq. 6  H_breve = H V I_f    (projection on the retained components).
 *   Eq. 7  M_breve_0(x, y) = sum_w |H_breve(x, y, w)|^2.
 *
 * Readings of the paper taken here (each is listed with its reason in the design notes):
 *  R1. Eq. 1 is written as a convolution but evaluated with one FFT. Expanding
 *      (x - x')^2 gives an input chirp exp(-i pi (x'^2)/(lambda z)), a DFT whose kernel
 *      is exp(+2 pi i x x'/(lambda z)) and an output chirp. The output chirp and the
 *      constant prefactor (i / lambda z) exp(-ikz) have unit modulus per pixel and
 *      cancel in C and in |H_breve|^2, so they are dropped. Input coordinates are
 *      centred (k - n/2). With a = pitch^2 / (lambda z) the discrete form is
 *        H[t,y,x] = s * sum_{k,l} I[t,l,k] c_x(k) c_y(l) exp(+2 pi i (x k / n_x + y l / n_y))
 *        c(k) = exp(-i pi a (k - n/2)^2),  s = 1 / sqrt(n_x n_y)  (unitary scale).
 *  R2. Eigenvalues are sorted in DEcreasing order and components are indexed from 0;
 *      the retained set is the inclusive range [k0, k1] of that order. (The paper
 *      sorts increasingly and counts from 1; its index j maps to k = n_t - j.)
 *      Ties keep the lower original index first.
 *  R3. "Complex-valued and symmetric" C (text before Eq. 4) is read as Hermitian, and
 *      the factorization of Eq. 5 as a Hermitian eigendecomposition.
 *  R4. Eq. 8's filter I_f keeps the diagonal entries n_1..n_2 counted, like the entries
 *      of W, from 1; here the temporal frequency bins are counted from 0, so the kept
 *      bins are k = n_1 - 1 .. n_2 - 1 (the paper's n_1 = 8, n_2 = 24 at n_t = 32 are
 *      bins 7..23).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define DHO_PI 3.14159265358979323846264338327950288

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int dho_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * 1-D complex DFT of length n (power of two), in place, unnormalised:
 *   X[m] = sum_k x[k] exp(sign * 2 pi i m k / n).
 * Iterative radix-2 (bit reversal, then butterflies). Twiddles are taken from
 * cos/sin of the exact angle at every use (no recurrence).
 * ------------------------------------------------------------------------- */
int dho_fft1d(int n, double *re, double *im, int sign) {
  if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j |= bit;
    if (i < j) {
      double tr = re[i]; re[i] = re[j]; re[j] = tr;
      double ti = im[i]; im[i] = im[j]; im[j] = ti;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len >> 1;
    for (int j = 0; j < half; ++j) {
      double ang = sign * 2.0 * DHO_PI * (double)j / (double)len;
      double wr = cos(ang), wi = sin(ang);
      for (int b = 0; b < n; b += len) {
        int u = b + j, v = b + j + half;
        double xr = re[v] * wr - im[v] * wi;
        double xi = re[v] * wi + im[v] * wr;
        re[v] = re[u] - xr; im[v] = im[u] - xi;
        re[u] += xr;        im[u] += xi;
      }
    }
  }
  return 0;
}

/* 2-D DFT of an ny x nx row-major array: rows, then columns. */
int dho_fft2d(int nx, int ny, double *re, double *im, int sign) {
  if (!is_pow2(nx) || !is_pow2(ny)) return -1;
  for (int y = 0; y < ny; ++y) dho_fft1d(nx, re + (size_t)y * nx, im + (size_t)y * nx, sign);
  double *cr = (double *)malloc(sizeof(double) * ny), *ci = (double *)malloc(sizeof(double) * ny);
  if (!cr || !ci) { free(cr); free(ci); return -2; }
  for (int x = 0; x < nx; ++x) {
    for (int y = 0; y < ny; ++y) { cr[y] = re[(size_t)y * nx + x]; ci[y] = im[(size_t)y * nx + x]; }
    dho_fft1d(ny, cr, ci, sign);
    for (int y = 0; y < ny; ++y) { re[(size_t)y * nx + x] = cr[y]; im[(size_t)y * nx + x] = ci[y]; }
  }
  free(cr); free(ci);
  return 0;
}

/* Input chirp of Eq. 1 (reading R1): c(k) = exp(-i pi a (k - n/2)^2), a = pitch^2/(lambda z).
 * The phase a (k - n/2)^2 is reduced modulo 2 before scaling by pi; (k - n/2)^2 is an
 * exact integer in double for every supported n. */
void dho_chirp(int n, double a, double *re, double *im) {
  for (int k = 0; k < n; ++k) {
    double d = (double)(k - n / 2);
    double ph = fmod(a * (d * d), 2.0);
    re[k] = cos(-DHO_PI * ph);
    im[k] = sin(-DHO_PI * ph);
  }
}

/* Eq. 1, reading R1: render T frames (uint16 [T][ny][nx]) into holograms H[T][ny][nx]. */
int dho_render(int nx, int ny, int T, const uint16_t *I, double lambda_m, double z_m,
               double pitch_m, double *Hre, double *Him) {
  if (!is_pow2(nx) || !is_pow2(ny) || T < 1 || !(lambda_m > 0) || !(z_m > 0) || !(pitch_m > 0))
    return -1;
  double a = pitch_m * pitch_m / (lambda_m * z_m);
  double *cxr = malloc(sizeof(double) * nx), *cxi = malloc(sizeof(double) * nx);
  double *cyr = malloc(sizeof(double) * ny), *cyi = malloc(sizeof(double) * ny);
  if (!cxr || !cxi || !cyr || !cyi) { free(cxr); free(cxi); free(cyr); free(cyi); return -2; }
  dho_chirp(nx, a, cxr, cxi);
  dho_chirp(ny, a, cyr, cyi);
  const size_t n = (size_t)nx * ny;
  const double s = 1.0 / sqrt((double)n);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int t = 0; t < T; ++t) {
    double *re = Hre + (size_t)t * n, *im = Him + (size_t)t * n;
    const uint16_t *src = I + (size_t)t * n;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double v = (double)src[(size_t)y * nx + x];
        /* v * c_x(x) * c_y(y) */
        double pr = cxr[x] * cyr[y] - cxi[x] * cyi[y];
        double pi = cxr[x] * cyi[y] + cxi[x] * cyr[y];
        re[(size_t)y * nx + x] = v * pr;
        im[(size_t)y * nx + x] = v * pi;
      }
    err |= dho_fft2d(nx, ny, re, im, +1);
    for (size_t p = 0; p < n; ++p) { re[p] *= s; im[p] *= s; }
  }
  free(cxr); free(cxi); free(cyr); free(cyi);
  return err;
}

/* Eq. 4: C = H^{t*} H, C[t][u] = sum_p conj(H[p][t]) H[p][u]. H is given frame-major
 * (H[t][p]); C is T x T, row-major re/im arrays. Pixels are summed in fixed blocks whose
 * partial matrices are added in block order, so the result does not depend on the
 * thread count. */
int dho_covariance(long long npix, int T, const double *Hre, const double *Him,
                   double *Cre, double *Cim) {
  if (npix < 1 || T < 1) return -1;
  const long long blk = 4096;
  const long long nblk = (npix + blk - 1) / blk;
  double *part = (double *)calloc((size_t)nblk * T * T * 2, sizeof(double));
  if (!part) return -2;
#pragma omp parallel for schedule(dynamic, 1)
  for (long long b = 0; b < nblk; ++b) {
    long long p0 = b * blk, p1 = p0 + blk < npix ? p0 + blk : npix;
    double *pr = part + (size_t)b * T * T * 2, *pi = pr + (size_t)T * T;
    for (int t = 0; t < T; ++t)
      for (int u = 0; u < T; ++u) {
        const double *ar = Hre + (size_t)t * npix, *ai = Him + (size_t)t * npix;
        const double *br = Hre + (size_t)u * npix, *bi = Him + (size_t)u * npix;
        double sr = 0.0, si = 0.0;
        for (long long p = p0; p < p1; ++p) {
          /* conj(a) * b */
          sr += ar[p] * br[p] + ai[p] * bi[p];
          si += ar[p] * bi[p] - ai[p] * br[p];
        }
        pr[t * T + u] = sr;
        pi[t * T + u] = si;
      }
  }
  memset(Cre, 0, sizeof(double) * T * T);
  memset(Cim, 0, sizeof(double) * T * T);
  for (long long b = 0; b < nblk; ++b) {
    const double *pr = part + (size_t)b * T * T * 2, *pi = pr + (size_t)T * T;
    for (int i = 0; i < T * T; ++i) { Cre[i] += pr[i]; Cim[i] += pi[i]; }
  }
  free(part);
  return 0;
}

/* Eq. 5: Hermitian eigendecomposition C = V Lambda V^{t*} by the cyclic two-sided
 * complex Jacobi method (row-cyclic order; Forsythe & Henrici 1960, Golub & Van Loan
 * Sec. 8.5). For a pair (p, q) with C_pq = g e^{i alpha}, the real symmetric 2x2 Schur
 * rotation (c, s) of [[C_pp, g], [g, C_qq]] is combined with the phase e^{i alpha}:
 *   J_pp = c, J_pq = s e^{i alpha}, J_qp = -s e^{-i alpha}, J_qq = c,
 * and C <- J^{t*} C J, V <- V J. Sweeps stop when the off-diagonal Frobenius norm is at
 * most tol * ||C||_F or after max_sweeps. Output: lam[T] sorted DEcreasing (reading R2)
 * and the matching unit eigenvectors as the columns of V (row-major V[t][k]).
 * Returns the number of sweeps used, or a negative value on error/non-convergence. */
int dho_eig(int T, const double *Cre, const double *Cim, double *lam, double *Vre,
            double *Vim, double tol, int max_sweeps) {
  if (T < 1) return -1;
  size_t TT = (size_t)T * T;
  double *ar = malloc(sizeof(double) * TT), *ai = malloc(sizeof(double) * TT);
  double *vr = malloc(sizeof(double) * TT), *vi = malloc(sizeof(double) * TT);
  double *d = malloc(sizeof(double) * T);
  int *order = malloc(sizeof(int) * T);
  if (!ar || !ai || !vr || !vi || !d || !order) {
    free(ar); free(ai); free(vr); free(vi); free(d); free(order); return -2;
  }
  memcpy(ar, Cre, sizeof(double) * TT);
  memcpy(ai, Cim, sizeof(double) * TT);
  /* Hermitian input: use the average of C and C^{t*} so the diagonal is real. */
  for (int i = 0; i < T; ++i)
    for (int j = i; j < T; ++j) {
      double r = 0.5 * (ar[i * T + j] + ar[j * T + i]);
      double m = 0.5 * (ai[i * T + j] - ai[j * T + i]);
      ar[i * T + j] = r; ai[i * T + j] = m;
      ar[j * T + i] = r; ai[j * T + i] = -m;
    }
  for (int i = 0; i < T; ++i) ai[i * T + i] = 0.0;
  memset(vr, 0, sizeof(double) * TT);
  memset(vi, 0, sizeof(double) * TT);
  for (int i = 0; i < T; ++i) vr[i * T + i] = 1.0;

  double fro = 0.0;
  for (size_t i = 0; i < TT; ++i) fro += ar[i] * ar[i] + ai[i] * ai[i];
  fro = sqrt(fro);
  int sweeps = 0, converged = 0;
  for (; sweeps <= max_sweeps; ++sweeps) {
    double off = 0.0;
    for (int i = 0; i < T; ++i)
      for (int j = 0; j < T; ++j)
        if (i != j) off += ar[i * T + j] * ar[i * T + j] + ai[i * T + j] * ai[i * T + j];
    if (sqrt(off) <= tol * fro) { converged = 1; break; }
    if (sweeps == max_sweeps) break;
    for (int p = 0; p < T - 1; ++p)
      for (int q = p + 1; q < T; ++q) {
        double gr = ar[p * T + q], gi = ai[p * T + q];
        double g = hypot(gr, gi);
        if (g == 0.0) continue;
        double er = gr / g, ei = gi / g; /* e^{i alpha} */
        double app = ar[p * T + p], aqq = ar[q * T + q];
        double tau = (aqq - app) / (2.0 * g);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* w = s e^{i alpha} */
        double wr = s * er, wi = s * ei;
        /* columns: A <- A J.  A_ip' = c A_ip - conj(w) A_iq ; A_iq' = w A_ip + c A_iq */
        for (int i = 0; i < T; ++i) {
          double xpr = ar[i * T + p], xpi = ai[i * T + p];
          double xqr = ar[i * T + q], xqi = ai[i * T + q];
          ar[i * T + p] = c * xpr - (wr * xqr + wi * xqi);
          ai[i * T + p] = c * xpi - (wr * xqi - wi * xqr);
          ar[i * T + q] = (wr * xpr - wi * xpi) + c * xqr;
          ai[i * T + q] = (wr * xpi + wi * xpr) + c * xqi;
        }
        /* rows: A <- J^{t*} A.  A_pj' = c A_pj - w A_qj ; A_qj' = conj(w) A_pj + c A_qj */
        for (int j = 0; j < T; ++j) {
          double xpr = ar[p * T + j], xpi = ai[p * T + j];
          double xqr = ar[q * T + j], xqi = ai[q * T + j];
          ar[p * T + j] = c * xpr - (wr * xqr - wi * xqi);
          ai[p * T + j] = c * xpi - (wr * xqi + wi * xqr);
          ar[q * T + j] = (wr * xpr + wi * xpi) + c * xqr;
          ai[q * T + j] = (wr * xpi - wi * xpr) + c * xqi;
        }
        ar[p * T + q] = ai[p * T + q] = 0.0;
        ar[q * T + p] = ai[q * T + p] = 0.0;
        ai[p * T + p] = ai[q * T + q] = 0.0;
        /* eigenvectors: V <- V J */
        for (int i = 0; i < T; ++i) {
          double xpr = vr[i * T + p], xpi = vi[i * T + p];
          double xqr = vr[i * T + q], xqi = vi[i * T + q];
          vr[i * T + p] = c * xpr - (wr * xqr + wi * xqi);
          vi[i * T + p] = c * xpi - (wr * xqi - wi * xqr);
          vr[i * T + q] = (wr * xpr - wi * xpi) + c * xqr;
          vi[i * T + q] = (wr * xpi + wi * xpr) + c * xqi;
        }
      }
  }
  for (int i = 0; i < T; ++i) { d[i] = ar[i * T + i]; order[i] = i; }
  /* reading R2: decreasing eigenvalues, ties by lower original index (stable insertion) */
  for (int i = 1; i < T; ++i) {
    int o = order[i], j = i - 1;
    while (j >= 0 && d[order[j]] < d[o]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = o;
  }
  for (int k = 0; k < T; ++k) {
    lam[k] = d[order[k]];
    for (int t = 0; t < T; ++t) {
      Vre[t * T + k] = vr[t * T + order[k]];
      Vim[t * T + k] = vi[t * T + order[k]];
    }
  }
  free(ar); free(ai); free(vr); free(vi); free(d); free(order);
  return converged ? sweeps : -3;
}

/* Eqs. 6-7: M[p] = sum_{k=k0..k1} |sum_t H[p][t] V[t][k]|^2 (reading R2 for k). */
int dho_project_power(long long npix, int T, const double *Hre, const double *Him,
                      const double *Vre, const double *Vim, int k0, int k1, double *M) {
  if (npix < 1 || T < 1 || k0 < 0 || k1 < k0 || k1 >= T) return -1;
#pragma omp parallel for schedule(static)
  for (long long p = 0; p < npix; ++p) {
    double acc = 0.0;
    for (int k = k0; k <= k1; ++k) {
      double pr = 0.0, pi = 0.0;
      for (int t = 0; t < T; ++t) {
        double hr = Hre[(size_t)t * npix + p], hi = Him[(size_t)t * npix + p];
        double v_r = Vre[t * T + k], v_i = Vim[t * T + k];
        pr += hr * v_r - hi * v_i;
        pi += hr * v_i + hi * v_r;
      }
      acc += pr * pr + pi * pi;
    }
    M[p] = acc;
  }
  return 0;
}

/* The whole window, in the paper's order: Eq. 1 -> Eq. 4 -> Eq. 5 -> Eqs. 6-7.
 * Outputs: M[ny*nx] (the image), lam[T] (decreasing), C (T x T re/im, optional: may be
 * NULL). Returns the Jacobi sweep count (>= 0) or a negative error. */
int dho_pca_window(int nx, int ny, int T, const uint16_t *I, double lambda_m, double z_m,
                   double pitch_m, int k0, int k1, double *M, double *lam, double *Cre_out,
                   double *Cim_out) {
  if (k0 < 0 || k1 < k0 || k1 >= T) return -1;
  size_t n = (size_t)nx * ny;
  double *hr = malloc(sizeof(double) * n * T), *hi = malloc(sizeof(double) * n * T);
  double *cr = malloc(sizeof(double) * T * T), *ci = malloc(sizeof(double) * T * T);
  double *vr = malloc(sizeof(double) * T * T), *vi = malloc(sizeof(double) * T * T);
  int rc = -2;
  if (hr && hi && cr && ci && vr && vi) {
    rc = dho_render(nx, ny, T, I, lambda_m, z_m, pitch_m, hr, hi);
    if (rc == 0) rc = dho_covariance((long long)n, T, hr, hi, cr, ci);
    if (rc == 0) {
      rc = dho_eig(T, cr, ci, lam, vr, vi, 1e-15, 60);
      if (rc >= 0) {
        int prc = dho_project_power((long long)n, T, hr, hi, vr, vi, k0, k1, M);
        if (prc != 0) rc = prc;
      }
    }
    if (Cre_out) memcpy(Cre_out, cr, sizeof(double) * T * T);
    if (Cim_out) memcpy(Cim_out, ci, sizeof(double) * T * T);
  }
  free(hr); free(hi); free(cr); free(ci); free(vr); free(vi);
  return rc;
}

/* Eqs. 8-9: temporal demodulation by the unitary DFT matrix W of Eq. 8,
 *   w_{t,k} = exp(-2 pi i t k / n_t) / sqrt(n_t)   (t, k counted from 0),
 * then the frequency filter and the power sum over the kept bins (reading R4):
 *   M[p] = sum_{k=k0..k1} |sum_t H[t][p] w_{t,k}|^2.
 * Written as the DFT's definition, O(n_t^2) per pixel; the angle is reduced exactly
 * (t k mod n_t) before the cosine and sine. */
int dho_fourier_power(long long npix, int T, const double *Hre, const double *Him, int k0,
                      int k1, double *M) {
  if (npix < 1 || T < 1 || k0 < 0 || k1 < k0 || k1 >= T) return -1;
  double *wr = malloc(sizeof(double) * T * T), *wi = malloc(sizeof(double) * T * T);
  if (!wr || !wi) { free(wr); free(wi); return -2; }
  const double s = 1.0 / sqrt((double)T);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < T; ++k) {
      const double ang = -2.0 * DHO_PI * (double)((t * k) % T) / (double)T;
      wr[t * T + k] = cos(ang) * s;
      wi[t * T + k] = sin(ang) * s;
    }
#pragma omp parallel for schedule(static)
  for (long long p = 0; p < npix; ++p) {
    double acc = 0.0;
    for (int k = k0; k <= k1; ++k) {
      double pr = 0.0, pi = 0.0;
      for (int t = 0; t < T; ++t) {
        double hr = Hre[(size_t)t * npix + p], hi = Him[(size_t)t * npix + p];
        pr += hr * wr[t * T + k] - hi * wi[t * T + k];
        pi += hr * wi[t * T + k] + hi * wr[t * T + k];
      }
      acc += pr * pr + pi * pi;
    }
    M[p] = acc;
  }
  free(wr); free(wi);
  return 0;
}

/* The Fourier-demodulated window, in the paper's order: Eq. 1 -> Eqs. 8-9. */
int dho_fourier_window(int nx, int ny, int T, const uint16_t *I, double lambda_m, double z_m,
                       double pitch_m, int k0, int k1, double *M) {
  if (k0 < 0 || k1 < k0 || k1 >= T) return -1;
  size_t n = (size_t)nx * ny;
  double *hr = malloc(sizeof(double) * n * T), *hi = malloc(sizeof(double) * n * T);
  int rc = -2;
  if (hr && hi) {
    rc = dho_render(nx, ny, T, I, lambda_m, z_m, pitch_m, hr, hi);
    if (rc == 0) rc = dho_fourier_power((long long)n, T, hr, hi, k0, k1, M);
  }
  free(hr); free(hi);
  return rc;
}

/* Eqs. 2-3 then Eqs. 8-9: singular value filtering of the window followed by temporal
 * demodulation by the unitary DFT, the paper's earlier (prior-art) pipeline.
 * Eq. 2 gives H = U Delta V^{t*}, so U Delta = H V with V the eigenvectors of C (Eq. 5),
 * and Eq. 3's filtered stack is H_f = U Delta I_f V^{t*} = (H V) I_f V^{t*}: for every pixel,
 *   P_k = sum_t H[t][p] V[t][k] for the kept components k = k0..k1 (reading R2),
 *   H_f[t][p] = sum_{k=k0..k1} P_k conj(V[t][k]),
 * then Eq. 8 with the filter of bins b0..b1 (reading R4) and Eq. 9:
 *   M[p] = sum_{b=b0..b1} |sum_t H_f[t][p] w_{t,b}|^2. */
int dho_svd_fourier_window(int nx, int ny, int T, const uint16_t *I, double lambda_m, double z_m,
                           double pitch_m, int k0, int k1, int b0, int b1, double *M,
                           double *lam) {
  if (k0 < 0 || k1 < k0 || k1 >= T || b0 < 0 || b1 < b0 || b1 >= T) return -1;
  size_t n = (size_t)nx * ny;
  double *hr = malloc(sizeof(double) * n * T), *hi = malloc(sizeof(double) * n * T);
  double *cr = malloc(sizeof(double) * T * T), *ci = malloc(sizeof(double) * T * T);
  double *vr = malloc(sizeof(double) * T * T), *vi = malloc(sizeof(double) * T * T);
  double *fr = malloc(sizeof(double) * n * T), *fi = malloc(sizeof(double) * n * T);
  int rc = -2;
  if (hr && hi && cr && ci && vr && vi && fr && fi) {
    rc = dho_render(nx, ny, T, I, lambda_m, z_m, pitch_m, hr, hi);
    if (rc == 0) rc = dho_covariance((long long)n, T, hr, hi, cr, ci);
    if (rc == 0) {
      rc = dho_eig(T, cr, ci, lam, vr, vi, 1e-15, 60);
      if (rc >= 0) {
#pragma omp parallel for schedule(static)
        for (long long p = 0; p < (long long)n; ++p) {
          for (int t = 0; t < T; ++t) { fr[(size_t)t * n + p] = 0.0; fi[(size_t)t * n + p] = 0.0; }
          for (int k = k0; k <= k1; ++k) {
            double pr = 0.0, pi = 0.0;
            for (int t = 0; t < T; ++t) {
              double a = hr[(size_t)t * n + p], b = hi[(size_t)t * n + p];
              pr += a * vr[t * T + k] - b * vi[t * T + k];
              pi += a * vi[t * T + k] + b * vr[t * T + k];
            }
            for (int t = 0; t < T; ++t) { /* P_k conj(V[t][k]) */
              fr[(size_t)t * n + p] += pr * vr[t * T + k] + pi * vi[t * T + k];
              fi[(size_t)t * n + p] += pi * vr[t * T + k] - pr * vi[t * T + k];
            }
          }
        }
        int frc = dho_fourier_power((long long)n, T, fr, fi, b0, b1, M);
        if (frc != 0) rc = frc;
      }
    }
  }
  free(hr); free(hi); free(cr); free(ci); free(vr); free(vi); free(fr); free(fi);
  return rc;
}
