// Eq. 4 (final FP64 reduction) and Eq. 5 on the GPU.
//
// k_reduce_cov: C[t][u] = sum over partial Gram matrices of
//     (G[2t][2u] + G[2t+1][2u+1]) + i (G[2t][2u+1] - G[2t+1][2u])   in FP64.
// k_jacobi: one CTA per window. Hermitian eigendecomposition C = V Lambda V^{t*} by the
//   two-sided complex Jacobi method (Forsythe & Henrici 1960; Golub & Van Loan Sec. 8.5)
//   with the parallel round-robin ordering: each of the T-1 steps of a sweep rotates T/2
//   disjoint pairs at once (Brent & Luk 1985); FP32 sweeps first, then refinement sweeps
//   from the Rayleigh quotient of the re-orthonormalised FP32 eigenvectors, in double-FP32
//   arithmetic with each rotation formed in FP64 (FP64 sweeps with DH_EIG_DF=0). For a pair with
//   C_pq = g e^{i alpha}, the real 2x2 Schur rotation (c, s) of [[C_pp, g], [g, C_qq]] is
//   combined with the phase: J_pp = J_qq = c, J_pq = s e^{i alpha}, J_qp = -s e^{-i alpha},
//   C <- J^{t*} C J, V <- V J. Eigenvalues are then ordered decreasing (ties by index)
//   and the retained columns k0..k1 are packed into the operand of Eq. 6.
#include "dh_internal.cuh"

// Refinement phase of the eigensolver: the off(A) / ||C||_F at which its sweeps stop, and its
// arithmetic (1: double-FP32, 0: FP64).
#ifndef DH_EIG_DF
#define DH_EIG_DF 1
#endif
#ifndef DH_EIG_TOL
#define DH_EIG_TOL 1e-12
#endif

namespace dh {
namespace {

template <int T>
__global__ void __launch_bounds__(256)
k_reduce_cov(const double *__restrict__ part, int parts, int n_windows, double *__restrict__ C,
             uint32_t *__restrict__ status) {
  constexpr int M = 2 * T;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_windows * T * T) return;
  const int w = idx / (T * T), e = idx % (T * T), t = e / T, u = e % T;
  const double *P = part + (long long)w * parts * M * M;
  double re = 0.0, im = 0.0;
  for (int q = 0; q < parts; ++q) {
    const double *G = P + (long long)q * M * M;
    re += G[(2 * t) * M + 2 * u] + G[(2 * t + 1) * M + 2 * u + 1];
    im += G[(2 * t) * M + 2 * u + 1] - G[(2 * t + 1) * M + 2 * u];
  }
  C[2 * ((long long)w * T * T + e)] = re;
  C[2 * ((long long)w * T * T + e) + 1] = im;
  if (!isfinite(re) || !isfinite(im)) atomicOr(status, DH_FLAG_NONFINITE_C);
}

// Raw-domain covariance: rows 2t / 2t+1 of the partial Gram matrices are the high / low bytes
// of frame t, so C[t][u] = sum over partials of 65536 G[2t][2u] + 256 (G[2t][2u+1] +
// G[2t+1][2u]) + G[2t+1][2u+1], all integers (exact in FP64 while below 2^53); Im C = 0.
template <int T>
__global__ void __launch_bounds__(256)
k_reduce_raw(const double *__restrict__ part, int parts, int n_windows, double *__restrict__ C,
             uint32_t *__restrict__ status) {
  constexpr int M = 2 * T;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_windows * T * T) return;
  const int w = idx / (T * T), e = idx % (T * T), t = e / T, u = e % T;
  const double *P = part + (long long)w * parts * M * M;
  double hh = 0.0, cross = 0.0, ll = 0.0;
  for (int q = 0; q < parts; ++q) {
    const double *G = P + (long long)q * M * M;
    hh += G[(2 * t) * M + 2 * u];
    cross += G[(2 * t) * M + 2 * u + 1] + G[(2 * t + 1) * M + 2 * u];
    ll += G[(2 * t + 1) * M + 2 * u + 1];
  }
  const double c = 65536.0 * hh + 256.0 * cross + ll;
  C[2 * ((long long)w * T * T + e)] = c;
  C[2 * ((long long)w * T * T + e) + 1] = 0.0;
  if (!isfinite(c)) atomicOr(status, DH_FLAG_NONFINITE_C);
}

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

template <typename T16> __device__ __forceinline__ T16 from_f32(float x);
template <> __device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <typename T16> __device__ __forceinline__ float to_f32(T16 x);
template <> __device__ __forceinline__ float to_f32<__half>(__half x) { return __half2float(x); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// Pack value v of operand entry (j, r) for the projection of Eq. 6 (see k_jacobi).
template <typename T16>
__device__ __forceinline__ void put_split(T16 *hi, T16 *lo, long long i, double v) {
  const T16 h = from_f32<T16>((float)v);
  hi[i] = h;
  lo[i] = from_f32<T16>((float)(v - (double)to_f32<T16>(h)));
}

// Upper-triangle element e (row-major, rows of T - i elements) -> (i, j), i <= j.
__device__ __forceinline__ void tri_ij(int e, int T, int &i, int &j) {
  const float b = 2.0f * T + 1.0f;
  int r = (int)((b - sqrtf(b * b - 8.0f * e)) * 0.5f);
  int start = r * T - r * (r - 1) / 2;
  if (start > e) { --r; start = r * T - r * (r - 1) / 2; }
  else if (start + (T - r) <= e) { start += T - r; ++r; }
  i = r;
  j = r + (e - start);
}

// Threads of the eigensolver's CTA: 512 at T = 64, where the FP64 phase has the most
// independent work per step and more warps keep the FP64 pipe busier; 256 below.
template <int T>
__host__ __device__ constexpr int kJacThreads() { return T == 64 ? 512 : 256; }

// Parallel-order two-sided complex Jacobi sweeps on the Hermitian matrix (ar, ai) (row
// stride LD), accumulating the rotations into (vr, vi). Real = float or double. Returns the
// number of sweeps taken, or -1 if off(A) > tol ||A||_F after max_sweeps.
template <int T, typename Real>
__device__ int jacobi_sweeps(Real *ar, Real *ai, Real *vr, Real *vi, double tol, int max_sweeps,
                             double fro, double *red) {
  constexpr int NP = T / 2;
  constexpr int LD = T + 1;
  __shared__ Real rc[NP], rwr[NP], rwi[NP];
  __shared__ int rp[NP], rq[NP];
  __shared__ unsigned short blk[NP * (NP + 1) / 2];  // pair blocks (P << 8 | Q), P <= Q
  const int tid = threadIdx.x;
  if constexpr (sizeof(Real) == 8 && T == 64) {
    for (int e = tid; e < NP * (NP + 1) / 2; e += blockDim.x) {
      int P, Q;
      tri_ij(e, NP, P, Q);
      blk[e] = (unsigned short)(P << 8 | Q);
    }
    __syncthreads();
  }
  const double inv_fro = fro > 0.0 ? 1.0 / fro : 0.0;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double off2;
    if constexpr (sizeof(Real) == 4) {  // a threshold test: FP32 on the entries over ||A||_F
      const float sc = (float)inv_fro;
      float o = 0.f;
      for (int e = tid; e < T * T; e += blockDim.x) {
        const int i = e / T, j = e % T;
        if (i != j) {
          const float x = (float)ar[i * LD + j] * sc, y = (float)ai[i * LD + j] * sc;
          o = fmaf(x, x, fmaf(y, y, o));
        }
      }
      off2 = block_sum((double)o, red) * fro * fro;
    } else {
      off2 = 0.0;
      for (int e = tid; e < T * T; e += blockDim.x) {
        const int i = e / T, j = e % T;
        if (i != j) {
          const double x = (double)ar[i * LD + j], y = (double)ai[i * LD + j];
          off2 += x * x + y * y;
        }
      }
      off2 = block_sum(off2, red);
    }
    if (sqrt(off2) <= tol * fro) return sweep;
    if (sweep == max_sweeps) break;
    for (int step = 0; step < T - 1; ++step) {
      if (tid < NP) {
        int a, b;
        if (tid == 0) { a = step; b = T - 1; }
        else { a = (step + tid) % (T - 1); b = (step - tid + T - 1) % (T - 1); }
        const int p = a < b ? a : b, q = a < b ? b : a;
        const Real gr = ar[p * LD + q], gi = ai[p * LD + q];
        Real c = 1, wr = 0, wi = 0;
        if constexpr (sizeof(Real) == 4) {
          const float g2 = gr * gr + gi * gi;
          if (g2 > (float)(1e-2 * tol * fro / T) * (float)(1e-2 * tol * fro / T)) {
            const float rg = rsqrtf(g2);
            const float tau = (ar[q * LD + q] - ar[p * LD + p]) * 0.5f * rg;
            const float t = __fdividef(copysignf(1.f, tau), fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            const float sn = t * c * rg;
            wr = sn * gr;
            wi = sn * gi;
          }
        } else {
        const Real g = sqrt(gr * gr + gi * gi);
        // rotations this small cannot hold off(A) above tol ||A||_F; they are skipped
        if (g > (Real)(1e-2 * tol * fro / T)) {
          const Real tau = (ar[q * LD + q] - ar[p * LD + p]) / (2 * g);
          const Real t = (tau >= 0 ? (Real)1 : (Real)-1) / (fabs(tau) + sqrt(1 + tau * tau));
          c = 1 / sqrt(1 + t * t);
          const Real sn = t * c;
          wr = sn * gr / g;
          wi = sn * gi / g;
        }
        }
        rp[tid] = p; rq[tid] = q; rc[tid] = c; rwr[tid] = wr; rwi[tid] = wi;
      }
      __syncthreads();
      if constexpr (sizeof(Real) == 4 || T < 64) {
        // FP32 (latency-bound), and FP64 below T = 64 (too little work per step for the block
        // form's bookkeeping to pay; measured): a column pass over A and V, then a row pass.
        // columns of A and V: X_ip' = c X_ip - conj(w) X_iq ;  X_iq' = w X_ip + c X_iq
        if constexpr (T == 64) {
          // FP32 at T = 64 (on the sliding and uneven workloads' critical path): a thread's four
          // items (k, i) share its row i and belong to distinct pairs, so they touch disjoint
          // elements; all their operands are loaded before any result is stored, which lets the
          // loads overlap (the arithmetic is unchanged). Measured: the sliding step's
          // eigensolver 5.65 -> 5.37 ms, the uneven step's 8.76 -> 8.26 ms. Below T = 64 the
          // loop is kept as it is (its CTA runs beside the other window group's covariance and
          // projection in the headline step, where a batched form measured slower for the whole
          // step). The kernel runs exactly kJacThreads<T>() threads.
          constexpr int NT = kJacThreads<T>(), IPT = NP * T / NT;
          static_assert(NP * T % NT == 0, "whole items per thread");
          Real xa[IPT][4], xv[IPT][4];
#pragma unroll
          for (int m = 0; m < IPT; ++m) {
            const int it = tid + m * NT, k = it / T, i = it % T, p = rp[k], q = rq[k];
            xa[m][0] = ar[i * LD + p]; xa[m][1] = ai[i * LD + p]; xa[m][2] = ar[i * LD + q]; xa[m][3] = ai[i * LD + q];
            xv[m][0] = vr[i * LD + p]; xv[m][1] = vi[i * LD + p]; xv[m][2] = vr[i * LD + q]; xv[m][3] = vi[i * LD + q];
          }
#pragma unroll
          for (int m = 0; m < IPT; ++m) {
            const int it = tid + m * NT, k = it / T, i = it % T;
            const Real c = rc[k], wr = rwr[k], wi = rwi[k];
            if (wr == 0 && wi == 0) continue;
            const int p = rp[k], q = rq[k];
            Real xpr = xa[m][0], xpi = xa[m][1], xqr = xa[m][2], xqi = xa[m][3];
            ar[i * LD + p] = c * xpr - (wr * xqr + wi * xqi);
            ai[i * LD + p] = c * xpi - (wr * xqi - wi * xqr);
            ar[i * LD + q] = (wr * xpr - wi * xpi) + c * xqr;
            ai[i * LD + q] = (wr * xpi + wi * xpr) + c * xqi;
            xpr = xv[m][0]; xpi = xv[m][1]; xqr = xv[m][2]; xqi = xv[m][3];
            vr[i * LD + p] = c * xpr - (wr * xqr + wi * xqi);
            vi[i * LD + p] = c * xpi - (wr * xqi - wi * xqr);
            vr[i * LD + q] = (wr * xpr - wi * xpi) + c * xqr;
            vi[i * LD + q] = (wr * xpi + wi * xpr) + c * xqi;
          }
        } else {
        for (int it = tid; it < NP * T; it += blockDim.x) {
          const int k = it / T, i = it % T;
          const Real c = rc[k], wr = rwr[k], wi = rwi[k];
          if (wr == 0 && wi == 0) continue;
          const int p = rp[k], q = rq[k];
          Real xpr = ar[i * LD + p], xpi = ai[i * LD + p], xqr = ar[i * LD + q], xqi = ai[i * LD + q];
          ar[i * LD + p] = c * xpr - (wr * xqr + wi * xqi);
          ai[i * LD + p] = c * xpi - (wr * xqi - wi * xqr);
          ar[i * LD + q] = (wr * xpr - wi * xpi) + c * xqr;
          ai[i * LD + q] = (wr * xpi + wi * xpr) + c * xqi;
          xpr = vr[i * LD + p]; xpi = vi[i * LD + p]; xqr = vr[i * LD + q]; xqi = vi[i * LD + q];
          vr[i * LD + p] = c * xpr - (wr * xqr + wi * xqi);
          vi[i * LD + p] = c * xpi - (wr * xqi - wi * xqr);
          vr[i * LD + q] = (wr * xpr - wi * xpi) + c * xqr;
          vi[i * LD + q] = (wr * xpi + wi * xpr) + c * xqi;
        }
        }
        __syncthreads();
        // rows of A: A_pj' = c A_pj - w A_qj ;  A_qj' = conj(w) A_pj + c A_qj. The pair's own
        // entries come out exact: A_pq = A_qp = 0 and real diagonal entries (also for a
        // skipped rotation, whose A_pq is below the skip level). At T = 64 a thread's items
        // (k, j) share its column j in distinct pairs: loads first, as in the column pass.
        if constexpr (T == 64) {
          constexpr int NT = kJacThreads<T>(), IPT = NP * T / NT;
          Real x4[IPT][4];
#pragma unroll
          for (int m = 0; m < IPT; ++m) {
            const int it = tid + m * NT, k = it / T, j = it % T, p = rp[k], q = rq[k];
            x4[m][0] = ar[p * LD + j]; x4[m][1] = ai[p * LD + j]; x4[m][2] = ar[q * LD + j]; x4[m][3] = ai[q * LD + j];
          }
#pragma unroll
          for (int m = 0; m < IPT; ++m) {
            const int it = tid + m * NT, k = it / T, j = it % T;
            const Real c = rc[k], wr = rwr[k], wi = rwi[k];
            const int p = rp[k], q = rq[k];
            if (wr == 0 && wi == 0) {
              if (j == p) { ai[p * LD + p] = 0; ar[q * LD + p] = ai[q * LD + p] = 0; }
              if (j == q) { ar[p * LD + q] = ai[p * LD + q] = 0; ai[q * LD + q] = 0; }
              continue;
            }
            const Real xpr = x4[m][0], xpi = x4[m][1], xqr = x4[m][2], xqi = x4[m][3];
            Real ypr = c * xpr - (wr * xqr - wi * xqi);
            Real ypi = c * xpi - (wr * xqi + wi * xqr);
            Real yqr = (wr * xpr + wi * xpi) + c * xqr;
            Real yqi = (wr * xpi - wi * xpr) + c * xqi;
            if (j == p) { ypi = 0; yqr = yqi = 0; }
            if (j == q) { ypr = ypi = 0; yqi = 0; }
            ar[p * LD + j] = ypr;
            ai[p * LD + j] = ypi;
            ar[q * LD + j] = yqr;
            ai[q * LD + j] = yqi;
          }
        } else {
        for (int it = tid; it < NP * T; it += blockDim.x) {
          const int k = it / T, j = it % T;
          const Real c = rc[k], wr = rwr[k], wi = rwi[k];
          const int p = rp[k], q = rq[k];
          if (wr == 0 && wi == 0) {
            if (j == p) { ai[p * LD + p] = 0; ar[q * LD + p] = ai[q * LD + p] = 0; }
            if (j == q) { ar[p * LD + q] = ai[p * LD + q] = 0; ai[q * LD + q] = 0; }
            continue;
          }
          const Real xpr = ar[p * LD + j], xpi = ai[p * LD + j], xqr = ar[q * LD + j], xqi = ai[q * LD + j];
          Real ypr = c * xpr - (wr * xqr - wi * xqi);
          Real ypi = c * xpi - (wr * xqi + wi * xqr);
          Real yqr = (wr * xpr + wi * xpi) + c * xqr;
          Real yqi = (wr * xpi - wi * xpr) + c * xqi;
          if (j == p) { ypi = 0; yqr = yqi = 0; }
          if (j == q) { ypr = ypi = 0; yqi = 0; }
          ar[p * LD + j] = ypr;
          ai[p * LD + j] = ypi;
          ar[q * LD + j] = yqr;
          ai[q * LD + j] = yqi;
        }
        }
        __syncthreads();
      } else {
        // FP64 at T = 64 (bound by the FP64 pipe): half the arithmetic on A (measured 13% off
        // the FP64 sweeps).
        // A <- K^H A K and V <- V K, K the T/2 disjoint rotations of this step: column op
        // x_p' = c x_p - conj(w) x_q, x_q' = w x_p + c x_q; row op the conjugate transpose.
        // A is Hermitian, so only the upper triangle of 2x2 pair blocks B(P,Q) =
        // A[{p_P, q_P}][{p_Q, q_Q}] (P <= Q) is updated, B -> B K_Q by rows (with V's columns),
        // then -> K_P^H (B K_Q) by columns, each block written with its mirror: every element of
        // A is computed once instead of once per pass.
        for (int it = tid; it < NP * (NP + 1) + NP * T; it += blockDim.x) {
          if (it < NP * (NP + 1)) {  // (block, row): B_r <- B_r K_Q
            const int P = blk[it >> 1] >> 8, Q = blk[it >> 1] & 255;
            const Real c = rc[Q], wr = rwr[Q], wi = rwi[Q];
            if (wr == 0 && wi == 0) continue;
            const int row = (it & 1) ? rq[P] : rp[P], p = rp[Q], q = rq[Q];
            const Real xpr = ar[row * LD + p], xpi = ai[row * LD + p], xqr = ar[row * LD + q], xqi = ai[row * LD + q];
            ar[row * LD + p] = c * xpr - (wr * xqr + wi * xqi);
            ai[row * LD + p] = c * xpi - (wr * xqi - wi * xqr);
            ar[row * LD + q] = (wr * xpr - wi * xpi) + c * xqr;
            ai[row * LD + q] = (wr * xpi + wi * xpr) + c * xqi;
          } else {  // columns of V
            const int k = (it - NP * (NP + 1)) / T, i = (it - NP * (NP + 1)) % T;
            const Real c = rc[k], wr = rwr[k], wi = rwi[k];
            if (wr == 0 && wi == 0) continue;
            const int p = rp[k], q = rq[k];
            const Real xpr = vr[i * LD + p], xpi = vi[i * LD + p], xqr = vr[i * LD + q], xqi = vi[i * LD + q];
            vr[i * LD + p] = c * xpr - (wr * xqr + wi * xqi);
            vi[i * LD + p] = c * xpi - (wr * xqi - wi * xqr);
            vr[i * LD + q] = (wr * xpr - wi * xpi) + c * xqr;
            vi[i * LD + q] = (wr * xpi + wi * xpr) + c * xqi;
          }
        }
        __syncthreads();
        for (int it = tid; it < NP * (NP + 1); it += blockDim.x) {  // (block, column): K_P^H B
          const int P = blk[it >> 1] >> 8, Q = blk[it >> 1] & 255;
          const Real c = rc[P], wr = rwr[P], wi = rwi[P];
          const bool rotP = !(wr == 0 && wi == 0);
          if (!rotP && !(rwr[Q] != 0 || rwi[Q] != 0)) continue;  // block unchanged
          const int cc = (it & 1) ? rq[Q] : rp[Q], r0 = rp[P], r1 = rq[P];
          const Real m0r = ar[r0 * LD + cc], m0i = ai[r0 * LD + cc], m1r = ar[r1 * LD + cc], m1i = ai[r1 * LD + cc];
          Real b0r = m0r, b0i = m0i, b1r = m1r, b1i = m1i;
          if (rotP) {  // row 0' = c M_0 - w M_1, row 1' = conj(w) M_0 + c M_1
            b0r = c * m0r - (wr * m1r - wi * m1i);
            b0i = c * m0i - (wr * m1i + wi * m1r);
            b1r = (wr * m0r + wi * m0i) + c * m1r;
            b1i = (wr * m0i - wi * m0r) + c * m1i;
          }
          if (P == Q) {  // the pair's own block: diagonal afterwards
            if ((it & 1) == 0) { b1r = 0; b1i = 0; b0i = 0; }
            else { b0r = 0; b0i = 0; b1i = 0; }
          }
          ar[r0 * LD + cc] = b0r; ai[r0 * LD + cc] = b0i;
          ar[r1 * LD + cc] = b1r; ai[r1 * LD + cc] = b1i;
          if (P != Q) {
            ar[cc * LD + r0] = b0r; ai[cc * LD + r0] = -b0i;
            ar[cc * LD + r1] = b1r; ai[cc * LD + r1] = -b1i;
          }
        }
        __syncthreads();
      }
    }
  }
  return -1;
}

// Eq. 5 for one window per CTA, in two precisions:
//  1. FP32 Jacobi sweeps on C until off(A) <= 1e-6 ||C||_F (the FP32 pipe is ~64x the FP64
//     pipe on this part);
//  2. FP64: the FP32 eigenvectors are re-orthonormalised (one second-order Lowdin step), C is
//     rotated into their basis (A = V^{t*} C V, the Rayleigh quotient), and FP64 Jacobi
//     sweeps finish A to off(A) <= tol ||C||_F, accumulating into V.
// The result is the FP64 eigendecomposition of C; phase 1 only supplies a good start.
// ---- double-FP32 ("df") arithmetic for the refinement phase. A value is h + l, two FP32
// numbers with |l| <= ulp(h)/2: a 48-bit significand. This part's FP64 pipe runs at about
// 1/100 of its FP32 rate, so the refinement's products and rotations are carried out with
// error-free transformations on FP32 (Knuth's TwoSum; the FMA-based exact product
// a b = p + fma(a, b, -p)), every operation an explicitly rounded intrinsic so that no
// contraction or reassociation changes it. Sums of products are accumulated unnormalised
// (h the running sum's leading part, l the collected errors) and normalised once at the end.
__device__ __forceinline__ float2 df_of(double d) {
  const float h = __double2float_rn(d);
  return make_float2(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double df_dbl(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_fin(float h, float l) {  // TwoSum(h, l)
  const float s = __fadd_rn(h, l);
  const float bb = __fsub_rn(s, h);
  return make_float2(s, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(l, bb)));
}
// (h, l) += a b
__device__ __forceinline__ void df_acc(float &h, float &l, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, e));
}
__device__ __forceinline__ float2 df_dot3(float2 a0, float2 b0, float2 a1, float2 b1, float2 a2, float2 b2) {
  float h = 0.f, l = 0.f;
  df_acc(h, l, a0, b0);
  df_acc(h, l, a1, b1);
  df_acc(h, l, a2, b2);
  return df_fin(h, l);
}
// sum_k op(a_k) b_k over k < T (op = conj when CONJ), complex df; a_k at index a0 + k sa,
// b_k at b0 + k sb of the re / im planes
template <int T, bool CONJ>
__device__ __forceinline__ void df_cdot(const float2 *ar, const float2 *ai, int a0, int sa, const float2 *br,
                                        const float2 *bi, int b0, int sb, float2 &outr, float2 &outi) {
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 4
  for (int k = 0; k < T; ++k) {
    const float2 xr_ = ar[a0 + k * sa], yr = br[b0 + k * sb], yi = bi[b0 + k * sb];
    const float2 xi_ = CONJ ? df_neg(ai[a0 + k * sa]) : ai[a0 + k * sa];
    df_acc(rh, rl, xr_, yr);
    df_acc(rh, rl, df_neg(xi_), yi);
    df_acc(ih, il, xr_, yi);
    df_acc(ih, il, xi_, yr);
  }
  outr = df_fin(rh, rl);
  outi = df_fin(ih, il);
}

// 1/sqrt(x) in FP64 from an estimate r0 within ~2^-22 (an FP32 reciprocal square root):
// two steps of Newton's iteration r <- r + r (1 - x r^2) / 2, each squaring the relative
// error, reach FP64 rounding
__device__ __forceinline__ double rsqrt_newton(double x, double r0) {
  double r = r0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double e = fma(-x * r, r, 1.0);
    r = fma(0.5 * r, e, r);
  }
  return r;
}

// Parallel-order complex Jacobi sweeps in df arithmetic on the Hermitian (ar, ai), rotations
// accumulated into (vr, vi); the rotation is formed in FP64 from the df entries (its tangent
// from an FP32 estimate).
// Same ordering, skip threshold and stopping rule as jacobi_sweeps.
template <int T>
__device__ int jacobi_sweeps_df(float2 *ar, float2 *ai, float2 *vr, float2 *vi, double tol, int max_sweeps,
                                double fro, double *red) {
  constexpr int NP = T / 2;
  constexpr int LD = T + 1;
  __shared__ float2 rc[NP], rwr[NP], rwi[NP];
  __shared__ int rp[NP], rq[NP], rskip[NP];
  __shared__ unsigned short blk[NP * (NP + 1) / 2];  // pair blocks (P << 8 | Q), P <= Q
  const int tid = threadIdx.x;
  if constexpr (T == 64) {
    for (int e = tid; e < NP * (NP + 1) / 2; e += blockDim.x) {
      int P, Q;
      tri_ij(e, NP, P, Q);
      blk[e] = (unsigned short)(P << 8 | Q);
    }
    __syncthreads();
  }
  const double inv_fro = fro > 0.0 ? 1.0 / fro : 0.0;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    // a threshold test: FP32 on the leading parts over ||A||_F (the trailing parts change
    // each square by less than 2^-23 of itself)
    const float sc = (float)inv_fro;
    float o = 0.f;
    for (int e = tid; e < T * T; e += blockDim.x) {
      const int i = e / T, j = e % T;
      if (i != j) {
        const float x = ar[i * LD + j].x * sc, y = ai[i * LD + j].x * sc;
        o = fmaf(x, x, fmaf(y, y, o));
      }
    }
    const double off2 = block_sum((double)o, red) * fro * fro;
    if (sqrt(off2) <= tol * fro) return sweep;
    if (sweep == max_sweeps) break;
    for (int step = 0; step < T - 1; ++step) {
      if (tid < NP) {
        int a, b;
        if (tid == 0) { a = step; b = T - 1; }
        else { a = (step + tid) % (T - 1); b = (step - tid + T - 1) % (T - 1); }
        const int p = a < b ? a : b, q = a < b ? b : a;
        const double gr = df_dbl(ar[p * LD + q]), gi = df_dbl(ai[p * LD + q]);
        const double g2 = gr * gr + gi * gi, thr = 1e-2 * tol * fro / T;
        double c = 1, wr = 0, wi = 0;
        int skip = 1;
        if (g2 > thr * thr) {  // smaller rotations cannot hold off(A) above tol ||A||_F
          // The tangent t in FP32, in units of ||A||_F (relative error ~1e-7: the rotation
          // leaves ~1e-7 of the entry, far below the stopping level after one sweep); then a
          // rotation unitary to FP64 rounding for that t: c = 1/sqrt(1 + t^2) and
          // w = t c g / |g|, both reciprocal square roots by Newton's iteration.
          // (g2s >= (1e-2 tol / T)^2: a normal FP32 value for tol >= 1e-15; the kernel runs
          // with tol = 1e-12)
          const float g2s = (float)(g2 * inv_fro * inv_fro);
          const float rgs = rsqrtf(g2s);
          const float tau = (float)((df_dbl(ar[q * LD + q]) - df_dbl(ar[p * LD + p])) * inv_fro) * 0.5f * rgs;
          const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
          const double td = (double)t;
          c = rsqrt_newton(fma(td, td, 1.0), (double)rsqrtf(fmaf(t, t, 1.f)));
          const double sn = td * c * rsqrt_newton(g2, (double)rgs * inv_fro);
          wr = sn * gr;
          wi = sn * gi;
          skip = 0;
        }
        rp[tid] = p; rq[tid] = q; rc[tid] = df_of(c); rwr[tid] = df_of(wr); rwi[tid] = df_of(wi);
        rskip[tid] = skip;
      }
      __syncthreads();
      if constexpr (T == 64) {  // measured: 8% off the sweeps at T = 64, none below
        // A <- K^H A K on the upper triangle of 2x2 pair blocks (P <= Q; rows of each block by
        // K_Q, with V's columns, then its columns by K_P^H, written with the mirror), so every
        // element of A is computed once; see jacobi_sweeps for the column and row operations.
        for (int it = tid; it < NP * (NP + 1) + NP * T; it += blockDim.x) {
          if (it < NP * (NP + 1)) {  // (block, row): B_r <- B_r K_Q
            const int P = blk[it >> 1] >> 8, Q = blk[it >> 1] & 255;
            if (rskip[Q]) continue;
            const float2 c = rc[Q], wr = rwr[Q], wi = rwi[Q];
            const int row = (it & 1) ? rq[P] : rp[P], p = rp[Q], q = rq[Q];
            const float2 xpr = ar[row * LD + p], xpi = ai[row * LD + p], xqr = ar[row * LD + q], xqi = ai[row * LD + q];
            ar[row * LD + p] = df_dot3(c, xpr, df_neg(wr), xqr, df_neg(wi), xqi);
            ai[row * LD + p] = df_dot3(c, xpi, df_neg(wr), xqi, wi, xqr);
            ar[row * LD + q] = df_dot3(wr, xpr, df_neg(wi), xpi, c, xqr);
            ai[row * LD + q] = df_dot3(wr, xpi, wi, xpr, c, xqi);
          } else {  // columns of V
            const int k = (it - NP * (NP + 1)) / T, i = (it - NP * (NP + 1)) % T;
            if (rskip[k]) continue;
            const float2 c = rc[k], wr = rwr[k], wi = rwi[k];
            const int p = rp[k], q = rq[k];
            const float2 xpr = vr[i * LD + p], xpi = vi[i * LD + p], xqr = vr[i * LD + q], xqi = vi[i * LD + q];
            vr[i * LD + p] = df_dot3(c, xpr, df_neg(wr), xqr, df_neg(wi), xqi);
            vi[i * LD + p] = df_dot3(c, xpi, df_neg(wr), xqi, wi, xqr);
            vr[i * LD + q] = df_dot3(wr, xpr, df_neg(wi), xpi, c, xqr);
            vi[i * LD + q] = df_dot3(wr, xpi, wi, xpr, c, xqi);
          }
        }
        __syncthreads();
        for (int it = tid; it < NP * (NP + 1); it += blockDim.x) {  // (block, column): K_P^H B
          const int P = blk[it >> 1] >> 8, Q = blk[it >> 1] & 255;
          if (rskip[P] && rskip[Q]) continue;  // block unchanged
          const int cc = (it & 1) ? rq[Q] : rp[Q], r0 = rp[P], r1 = rq[P];
          float2 b0r = ar[r0 * LD + cc], b0i = ai[r0 * LD + cc], b1r = ar[r1 * LD + cc], b1i = ai[r1 * LD + cc];
          if (!rskip[P]) {  // row 0' = c M_0 - w M_1, row 1' = conj(w) M_0 + c M_1
            const float2 c = rc[P], wr = rwr[P], wi = rwi[P];
            const float2 m0r = b0r, m0i = b0i, m1r = b1r, m1i = b1i;
            b0r = df_dot3(c, m0r, df_neg(wr), m1r, wi, m1i);
            b0i = df_dot3(c, m0i, df_neg(wr), m1i, df_neg(wi), m1r);
            b1r = df_dot3(wr, m0r, wi, m0i, c, m1r);
            b1i = df_dot3(wr, m0i, df_neg(wi), m0r, c, m1i);
          }
          if (P == Q) {  // the pair's own block: diagonal afterwards
            const float2 z = make_float2(0.f, 0.f);
            if ((it & 1) == 0) { b1r = z; b1i = z; b0i = z; }
            else { b0r = z; b0i = z; b1i = z; }
          }
          ar[r0 * LD + cc] = b0r; ai[r0 * LD + cc] = b0i;
          ar[r1 * LD + cc] = b1r; ai[r1 * LD + cc] = b1i;
          if (P != Q) {
            ar[cc * LD + r0] = b0r; ai[cc * LD + r0] = df_neg(b0i);
            ar[cc * LD + r1] = b1r; ai[cc * LD + r1] = df_neg(b1i);
          }
        }
        __syncthreads();
      } else {
        // columns of A and V: X_ip' = c X_ip - conj(w) X_iq ;  X_iq' = w X_ip + c X_iq
        for (int it = tid; it < 2 * NP * T; it += blockDim.x) {
          const bool isv = it >= NP * T;
          const int k = (isv ? it - NP * T : it) / T, i = (isv ? it - NP * T : it) % T;
          if (rskip[k]) continue;
          const float2 c = rc[k], wr = rwr[k], wi = rwi[k];
          float2 *xr_ = isv ? vr : ar, *xi_ = isv ? vi : ai;
          const int p = rp[k], q = rq[k];
          const float2 xpr = xr_[i * LD + p], xpi = xi_[i * LD + p], xqr = xr_[i * LD + q], xqi = xi_[i * LD + q];
          xr_[i * LD + p] = df_dot3(c, xpr, df_neg(wr), xqr, df_neg(wi), xqi);
          xi_[i * LD + p] = df_dot3(c, xpi, df_neg(wr), xqi, wi, xqr);
          xr_[i * LD + q] = df_dot3(wr, xpr, df_neg(wi), xpi, c, xqr);
          xi_[i * LD + q] = df_dot3(wr, xpi, wi, xpr, c, xqi);
        }
        __syncthreads();
        // rows of A: A_pj' = c A_pj - w A_qj ;  A_qj' = conj(w) A_pj + c A_qj; a rotated
        // pair's own entries come out exact (A_pq = A_qp = 0, real diagonal entries)
        for (int it = tid; it < NP * T; it += blockDim.x) {
          const int k = it / T, j = it % T;
          if (rskip[k]) continue;
          const float2 c = rc[k], wr = rwr[k], wi = rwi[k];
          const int p = rp[k], q = rq[k];
          const float2 xpr = ar[p * LD + j], xpi = ai[p * LD + j], xqr = ar[q * LD + j], xqi = ai[q * LD + j];
          const float2 z = make_float2(0.f, 0.f);
          float2 ypr = df_dot3(c, xpr, df_neg(wr), xqr, wi, xqi);
          float2 ypi = df_dot3(c, xpi, df_neg(wr), xqi, df_neg(wi), xqr);
          float2 yqr = df_dot3(wr, xpr, wi, xpi, c, xqr);
          float2 yqi = df_dot3(wr, xpi, df_neg(wi), xpr, c, xqi);
          if (j == p) { ypi = z; yqr = z; yqi = z; }
          if (j == q) { ypr = z; ypi = z; yqi = z; }
          ar[p * LD + j] = ypr; ai[p * LD + j] = ypi;
          ar[q * LD + j] = yqr; ai[q * LD + j] = yqi;
        }
        __syncthreads();
      }
    }
  }
  return -1;
}

template <int T>
__global__ void __launch_bounds__(kJacThreads<T>())
k_jacobi(const double *__restrict__ C, double *__restrict__ lam, double *__restrict__ Vout,
         double *__restrict__ eig_user, int prec, void *__restrict__ Bop, long long B_stride,
         int k0, int k1, int Npad, double tol, int max_sweeps, uint32_t *__restrict__ status) {
  constexpr int LD = T + 1;
  constexpr int M = 2 * T;
  constexpr int SZ = T * LD;
  extern __shared__ double sm[];
  // X: C, later A (FP64); Y: V (FP64); Z: FP32 A and V in phase 1, FP64 scratch in phase 2
  double *xr = sm, *xi = xr + SZ, *vr = xi + SZ, *vi = vr + SZ, *zr = vi + SZ, *zi = zr + SZ;
  float *ar32 = reinterpret_cast<float *>(zr), *ai32 = ar32 + SZ, *vr32 = ai32 + SZ, *vi32 = vr32 + SZ;
  __shared__ double red[16], dsort[T];
  __shared__ int perm[T];
  const int w = blockIdx.x, tid = threadIdx.x;
  const double *Cw = C + 2ll * w * T * T;

  double fro2 = 0.0;
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T;
    const double re = 0.5 * (Cw[2 * (i * T + j)] + Cw[2 * (j * T + i)]);
    const double im = i == j ? 0.0 : 0.5 * (Cw[2 * (i * T + j) + 1] - Cw[2 * (j * T + i) + 1]);
    xr[i * LD + j] = re;
    xi[i * LD + j] = im;
    ar32[i * LD + j] = (float)re;
    ai32[i * LD + j] = (float)im;
    vr32[i * LD + j] = i == j ? 1.f : 0.f;
    vi32[i * LD + j] = 0.f;
    fro2 += re * re + im * im;
  }
  const double fro = sqrt(block_sum(fro2, red));

  // ---- phase 1: FP32
  jacobi_sweeps<T, float>(ar32, ai32, vr32, vi32, 1e-6, 20, fro, red);

#if DH_EIG_DF
  // ---- phase 2: double-FP32 refinement (see df_acc); C, V and A in df form in the same
  // 8-byte slots as the FP64 arrays, converted back to FP64 at the end
  {
    constexpr int NTRI = T * (T + 1) / 2;
    constexpr int NT = kJacThreads<T>();
    constexpr int TPT = (NTRI + NT - 1) / NT;  // upper-triangle elements per thread
    float2 *XR = reinterpret_cast<float2 *>(xr), *XI = reinterpret_cast<float2 *>(xi);
    float2 *VR = reinterpret_cast<float2 *>(vr), *VI = reinterpret_cast<float2 *>(vi);
    float2 *ZR = reinterpret_cast<float2 *>(zr), *ZI = reinterpret_cast<float2 *>(zi);
    for (int e = tid; e < T * T; e += blockDim.x) {
      const int i = e / T, j = e % T;
      const float a = vr32[i * LD + j], b = vi32[i * LD + j];  // read before the C slots change
      VR[i * LD + j] = make_float2(a, 0.f);
      VI[i * LD + j] = make_float2(b, 0.f);
      XR[i * LD + j] = df_of(xr[i * LD + j]);
      XI[i * LD + j] = df_of(xi[i * LD + j]);
    }
    __syncthreads();
    // Lowdin re-orthonormalisation, second order in one step: E = V^{t*} V - I (Hermitian,
    // |E| ~ 1e-6 after the FP32 sweeps), V <- V (I - E/2 + 3E^2/8), orthogonality error
    // O(|E|^3). Y's small terms are formed in FP64.
    for (int e = tid; e < NTRI; e += blockDim.x) {
      int i, j;
      tri_ij(e, T, i, j);
      float2 sr, si;
      df_cdot<T, true>(VR, VI, i, LD, VR, VI, j, LD, sr, si);
      if (i == j) { sr = df_of(df_dbl(sr) - 1.0); si = make_float2(0.f, 0.f); }
      ZR[i * LD + j] = sr; ZI[i * LD + j] = si;
      ZR[j * LD + i] = sr; ZI[j * LD + i] = df_neg(si);
    }
    __syncthreads();
    {
      double yr[TPT], yi[TPT];
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        const int e = tid + u * NT;
        yr[u] = yi[u] = 0.0;
        if (e < NTRI) {
          int i, j;
          tri_ij(e, T, i, j);
          float2 sr, si;  // (E^2)_ij
          df_cdot<T, false>(ZR, ZI, i * LD, 1, ZR, ZI, j, LD, sr, si);
          yr[u] = (i == j ? 1.0 : 0.0) - 0.5 * df_dbl(ZR[i * LD + j]) + 0.375 * df_dbl(sr);
          yi[u] = -0.5 * df_dbl(ZI[i * LD + j]) + 0.375 * df_dbl(si);
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        const int e = tid + u * NT;
        if (e < NTRI) {
          int i, j;
          tri_ij(e, T, i, j);
          ZR[i * LD + j] = df_of(yr[u]); ZI[i * LD + j] = i == j ? make_float2(0.f, 0.f) : df_of(yi[u]);
          ZR[j * LD + i] = df_of(yr[u]); ZI[j * LD + i] = i == j ? make_float2(0.f, 0.f) : df_of(-yi[u]);
        }
      }
      __syncthreads();
    }
    {  // V <- V Y: thread (row i, CPT columns)
      constexpr int NPR = NT / T;
      constexpr int CPT = T / NPR;
      const int i = tid / NPR, j0 = (tid % NPR) * CPT;
      float rh[CPT], rl[CPT], ih[CPT], il[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) rh[c] = rl[c] = ih[c] = il[c] = 0.f;
      if (i < T) {
        for (int k = 0; k < T; ++k) {
          const float2 ar_ = VR[i * LD + k], ai_ = VI[i * LD + k];
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const float2 br = ZR[k * LD + j0 + c], bi = ZI[k * LD + j0 + c];
            df_acc(rh[c], rl[c], ar_, br);
            df_acc(rh[c], rl[c], df_neg(ai_), bi);
            df_acc(ih[c], il[c], ar_, bi);
            df_acc(ih[c], il[c], ai_, br);
          }
        }
      }
      __syncthreads();
      if (i < T) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          VR[i * LD + j0 + c] = df_fin(rh[c], rl[c]);
          VI[i * LD + j0 + c] = df_fin(ih[c], il[c]);
        }
      }
      __syncthreads();
    }
    // Rayleigh quotient A = V^{t*} (C V): Z = C V in full, then A's upper triangle (Hermitian)
    for (int e = tid; e < T * T; e += blockDim.x) {
      const int i = e / T, j = e % T;
      float2 sr, si;
      df_cdot<T, false>(XR, XI, i * LD, 1, VR, VI, j, LD, sr, si);
      ZR[i * LD + j] = sr; ZI[i * LD + j] = si;
    }
    __syncthreads();
    for (int e = tid; e < NTRI; e += blockDim.x) {
      int i, j;
      tri_ij(e, T, i, j);
      float2 sr, si;
      df_cdot<T, true>(VR, VI, i, LD, ZR, ZI, j, LD, sr, si);
      if (i == j) si = make_float2(0.f, 0.f);
      XR[i * LD + j] = sr; XI[i * LD + j] = si;
      XR[j * LD + i] = sr; XI[j * LD + i] = df_neg(si);
    }
    __syncthreads();
    const int sweeps = jacobi_sweeps_df<T>(XR, XI, VR, VI, tol, max_sweeps, fro, red);
    if (sweeps < 0 && tid == 0) atomicOr(status, DH_FLAG_EIG_NOT_CONVERGED);
    // back to FP64 in place (each slot read and written by the same thread)
    for (int e = tid; e < T * T; e += blockDim.x) {
      const int i = e / T, j = e % T;
      const double a = df_dbl(XR[i * LD + j]), b = df_dbl(VR[i * LD + j]), c = df_dbl(VI[i * LD + j]);
      xr[i * LD + j] = a;
      vr[i * LD + j] = b;
      vi[i * LD + j] = c;
    }
    __syncthreads();
  }
#else
  // ---- phase 2: FP64
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T;
    vr[i * LD + j] = (double)vr32[i * LD + j];
    vi[i * LD + j] = (double)vi32[i * LD + j];
  }
  __syncthreads();
  // Lowdin re-orthonormalisation of the (nearly orthonormal) columns of V, second order in
  // one pass: with E = V^{t*} V - I (|E| ~ 1e-6 after the FP32 sweeps),
  // (V^{t*} V)^{-1/2} = I - E/2 + 3E^2/8 - ..., so V <- V (I - E/2 + 3E^2/8) leaves an
  // orthogonality error O(|E|^3), below FP64 rounding. E and E^2 are Hermitian: only their
  // upper triangles are computed.
  constexpr int NTRI = T * (T + 1) / 2;
  constexpr int NT = kJacThreads<T>();
  constexpr int TPT = (NTRI + NT - 1) / NT;  // upper-triangle elements per thread
  for (int e = tid; e < NTRI; e += blockDim.x) {  // Z = E = V^{t*} V - I
    int i, j;
    tri_ij(e, T, i, j);
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < T; ++k) {
      const double ar_ = vr[k * LD + i], ai_ = -vi[k * LD + i], br = vr[k * LD + j], bi = vi[k * LD + j];
      sr += ar_ * br - ai_ * bi;
      si += ar_ * bi + ai_ * br;
    }
    if (i == j) { sr -= 1.0; si = 0.0; }
    zr[i * LD + j] = sr; zi[i * LD + j] = si;
    zr[j * LD + i] = sr; zi[j * LD + i] = -si;
  }
  __syncthreads();
  {
    double yr[TPT], yi[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int e = tid + u * NT;
      yr[u] = yi[u] = 0.0;
      if (e < NTRI) {
        int i, j;
        tri_ij(e, T, i, j);
        double sr = 0.0, si = 0.0;  // (E^2)_ij
        for (int k = 0; k < T; ++k) {
          const double ar_ = zr[i * LD + k], ai_ = zi[i * LD + k], br = zr[k * LD + j], bi = zi[k * LD + j];
          sr += ar_ * br - ai_ * bi;
          si += ar_ * bi + ai_ * br;
        }
        yr[u] = (i == j ? 1.0 : 0.0) - 0.5 * zr[i * LD + j] + 0.375 * sr;
        yi[u] = -0.5 * zi[i * LD + j] + 0.375 * si;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int e = tid + u * NT;
      if (e < NTRI) {
        int i, j;
        tri_ij(e, T, i, j);
        zr[i * LD + j] = yr[u]; zi[i * LD + j] = i == j ? 0.0 : yi[u];
        zr[j * LD + i] = yr[u]; zi[j * LD + i] = i == j ? 0.0 : -yi[u];
      }
    }
    __syncthreads();
  }
  {  // V <- V Y
    constexpr int NPR = NT / T;    // threads per row of V
    constexpr int CPT = T / NPR;   // output columns per thread
    const int i = tid / NPR, j0 = (tid % NPR) * CPT;
    double nr[CPT], ni[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) nr[c] = 0.0, ni[c] = 0.0;
    if (i < T) {
      for (int k = 0; k < T; ++k) {
        const double ar_ = vr[i * LD + k], ai_ = vi[i * LD + k];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const double br = zr[k * LD + j0 + c], bi = zi[k * LD + j0 + c];
          nr[c] += ar_ * br - ai_ * bi;
          ni[c] += ar_ * bi + ai_ * br;
        }
      }
    }
    __syncthreads();
    if (i < T) {
#pragma unroll
      for (int c = 0; c < CPT; ++c) { vr[i * LD + j0 + c] = nr[c]; vi[i * LD + j0 + c] = ni[c]; }
    }
    __syncthreads();
  }

  // Z = C V
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T;
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < T; ++k) {
      const double cr = xr[i * LD + k], ci = xi[i * LD + k], br = vr[k * LD + j], bi = vi[k * LD + j];
      sr += cr * br - ci * bi;
      si += cr * bi + ci * br;
    }
    zr[i * LD + j] = sr;
    zi[i * LD + j] = si;
  }
  __syncthreads();
  // X = V^{t*} Z, Hermitian: the upper triangle, mirrored (C is not needed any more)
  for (int e = tid; e < NTRI; e += blockDim.x) {
    int i, j;
    tri_ij(e, T, i, j);
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < T; ++k) {
      const double ar_ = vr[k * LD + i], ai_ = -vi[k * LD + i], br = zr[k * LD + j], bi = zi[k * LD + j];
      sr += ar_ * br - ai_ * bi;
      si += ar_ * bi + ai_ * br;
    }
    if (i == j) si = 0.0;
    xr[i * LD + j] = sr; xi[i * LD + j] = si;
    xr[j * LD + i] = sr; xi[j * LD + i] = -si;
  }
  __syncthreads();
  const int sweeps = jacobi_sweeps<T, double>(xr, xi, vr, vi, tol, max_sweeps, fro, red);
  if (sweeps < 0 && tid == 0) atomicOr(status, DH_FLAG_EIG_NOT_CONVERGED);

#endif

  // decreasing order, ties by original index. A NaN (from a non-finite C, which the covariance
  // reduction flags) orders after every number, so that the ranks are a permutation whatever
  // the values and every index taken from perm below stays in [0, T).
  if (tid < T) dsort[tid] = xr[tid * LD + tid];
  __syncthreads();
  if (tid < T) {
    auto key = [](double x) { return isnan(x) ? -INFINITY : x; };
    const double d = key(dsort[tid]);
    int rank = 0;
    for (int j = 0; j < T; ++j) {
      const double x = key(dsort[j]);
      rank += (x > d) || (x == d && j < tid);
    }
    perm[rank] = tid;
  }
  __syncthreads();
  if (tid < T) {
    lam[(long long)w * T + tid] = dsort[perm[tid]];
    if (eig_user) eig_user[(long long)w * T + tid] = dsort[perm[tid]];
  }
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int t = e / T, k = e % T;
    Vout[2 * ((long long)w * T * T + e)] = vr[t * LD + perm[k]];
    Vout[2 * ((long long)w * T * T + e) + 1] = vi[t * LD + perm[k]];
  }
  // Operand of Eq. 6 in the real embedding [P_re P_im] = [Re H, Im H] * B^T, rows r = 2t + c:
  //   j < nS       (P_re of component k = k0 + j):  B[j][2t] = Re V_tk, B[j][2t+1] = -Im V_tk
  //   nS <= j < 2nS (P_im of k = k0 + j - nS):      B[j][2t] = Im V_tk, B[j][2t+1] =  Re V_tk
  const int nS = k1 - k0 + 1;
  for (int e = tid; e < Npad * M; e += blockDim.x) {
    const int j = e / M, r = e % M, t = r >> 1, c = r & 1;
    double v = 0.0;
    if (j < 2 * nS) {
      const int k = k0 + (j < nS ? j : j - nS);
      const double re = vr[t * LD + perm[k]], im = vi[t * LD + perm[k]];
      v = j < nS ? (c == 0 ? re : -im) : (c == 0 ? im : re);
    }
    if (prec == DH_PREC_FP32) {
      static_cast<float *>(Bop)[w * B_stride + e] = (float)v;
    } else if (prec == DH_PREC_FP16) {
      __half *hi = static_cast<__half *>(Bop) + w * B_stride;
      put_split<__half>(hi, hi + (long long)Npad * M, e, v);
    } else {
      __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(Bop) + w * B_stride;
      put_split<__nv_bfloat16>(hi, hi + (long long)Npad * M, e, v);
    }
  }
}

// Operand of the grouped projection of overlapping windows (csrc/project_span.cu): window w's
// CPW columns of its group's banded operand (group of G windows, slot stride s), from its
// sorted eigenvectors V (FP64, [T][T] re/im). Column 2d + c of the window holds discarded
// component d (k < k0 first, then k > k1; zero past the last) as the real embedding row of
// Eq. 6 (c = 0: Re, c = 1: Im) at span rows 2 (s g + t) + {0, 1}, zeros elsewhere; stored as
// hi + lo 16-bit images of n_pad x k_pad in the K-major 128-byte-swizzled order the tensor
// cores read (64-element sub-blocks; the 16-byte chunk index XOR row % 8). The values are
// scaled by 2^10 (kSpanOperandScale) so that the lo part of an entry near 1/sqrt(T) stays a
// normal FP16 number: unscaled, it falls below 2^-14 and keeps only a few bits, which limits
// V to ~21 bits; the projection multiplies the squared products back by 2^-20, exactly.
__global__ void k_span_operand(const double *__restrict__ V, int T, int n_windows, int k0, int k1, SpanLayout sp,
                               int bf16, void *__restrict__ Bop, long long B_stride) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = sp.cpw * sp.k_pad;
  if (idx >= n_windows * per) return;
  const int w = idx / per, e = idx % per;
  const int g = w % sp.G;
  const int nD = k0 + (T - 1 - k1);
  const int nl = e / sp.k_pad, r = e % sp.k_pad;
  const int d = nl >> 1, c = nl & 1;                 // discarded component d; Re / Im column
  const int t = (r >> 1) - sp.stride * g, cc = r & 1;  // window frame t; Re / Im row
  double v = 0.0;
  if (d < nD && t >= 0 && t < T) {
    const int k = d < k0 ? d : k1 + 1 + (d - k0);
    const double re = V[2 * ((long long)w * T * T + t * T + k)], im = V[2 * ((long long)w * T * T + t * T + k) + 1];
    v = (c == 0 ? (cc == 0 ? re : -im) : (cc == 0 ? im : re)) * kSpanOperandScale;
  }
  const int n = g * sp.cpw + nl, sub = r >> 6, kk = r & 63;
  const long long i =
      ((long long)sub * sp.n_pad * 128 + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + ((kk & 7) << 1)) >> 1;
  const long long img = (long long)sp.n_pad * sp.k_pad;  // elements of one of hi / lo
  if (bf16) {
    __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(Bop) + (long long)(w - g) * B_stride;
    put_split<__nv_bfloat16>(hi, hi + img, i, v);
  } else {
    __half *hi = static_cast<__half *>(Bop) + (long long)(w - g) * B_stride;
    put_split<__half>(hi, hi + img, i, v);
  }
}

template <int T>
dh_status launch_reduce_t(Plan &p, int n_windows, int parts, int woff, cudaStream_t s) {
  const int total = n_windows * T * T;
  ProfScope ps(p, K_REDUCE_COV, s);
  k_reduce_cov<T><<<(total + 255) / 256, 256, 0, s>>>(p.d_part, parts, n_windows,
                                                      p.d_C + 2ll * woff * T * T, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

template <int T>
dh_status launch_jacobi_t(Plan &p, int n_windows, int k0, int k1, int Npad, double *eig_user, int woff,
                          cudaStream_t s, const SpanLayout *span) {
  if (span) Npad = 0;  // the grouped projection's operand is written below instead
  const size_t smem = 6ull * T * (T + 1) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(k_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long B_stride = (long long)(p.B_window_bytes / (p.prec == DH_PREC_FP32 ? 4 : 2));
  void *B = static_cast<char *>(p.d_B) + (size_t)woff * p.B_window_bytes;
  ProfScope ps(p, K_JACOBI, s);
  k_jacobi<T><<<n_windows, kJacThreads<T>(), smem, s>>>(p.d_C + 2ll * woff * T * T, p.d_lam + (long long)woff * T,
                                           p.d_V + 2ll * woff * T * T, eig_user, (int)p.prec, B, B_stride,
                                           k0, k1, Npad, DH_EIG_TOL, 30, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  if (span) {
    const int total = n_windows * span->cpw * span->k_pad;
    const long long B_stride = (long long)(p.B_window_bytes / 2);
    void *B = static_cast<char *>(p.d_B) + (size_t)woff * p.B_window_bytes;
    k_span_operand<<<(total + 255) / 256, 256, 0, s>>>(p.d_V + 2ll * woff * T * T, T, n_windows, k0, k1,
                                                       *span, p.prec == DH_PREC_BF16, B, B_stride);
    DH_CUDA_TRY(cudaGetLastError());
  }
  return DH_OK;
}

}  // namespace

// FP64 sum of `parts` partial Gram matrices of one window into C (T x T, interleaved re/im).
dh_status launch_reduce_cov_window(const double *part, int parts, int T, double *C, uint32_t *status,
                                   cudaStream_t s) {
  const int blocks = (T * T + 255) / 256;
  switch (T) {
    case 16: k_reduce_cov<16><<<blocks, 256, 0, s>>>(part, parts, 1, C, status); break;
    case 32: k_reduce_cov<32><<<blocks, 256, 0, s>>>(part, parts, 1, C, status); break;
    case 64: k_reduce_cov<64><<<blocks, 256, 0, s>>>(part, parts, 1, C, status); break;
    default: return DH_ERR_UNSUPPORTED_SIZE;
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

// Loads the module of every instance launch_reduce_cov_window uses (see preload_gram_simt_rows).
dh_status preload_reduce_cov_window() {
  cudaFuncAttributes fa;
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, k_reduce_cov<16>));
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, k_reduce_cov<32>));
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, k_reduce_cov<64>));
  return DH_OK;
}

dh_status launch_reduce_raw(Plan &p, int n_windows, int parts, int woff, cudaStream_t s) {
  const int total = n_windows * p.T * p.T;
  ProfScope ps(p, K_REDUCE_RAW, s);
  switch (p.T) {
    case 16: k_reduce_raw<16><<<(total + 255) / 256, 256, 0, s>>>(p.d_part, parts, n_windows,
                                                                  p.d_C + 2ll * woff * 16 * 16, p.d_status); break;
    case 32: k_reduce_raw<32><<<(total + 255) / 256, 256, 0, s>>>(p.d_part, parts, n_windows,
                                                                  p.d_C + 2ll * woff * 32 * 32, p.d_status); break;
    case 64: k_reduce_raw<64><<<(total + 255) / 256, 256, 0, s>>>(p.d_part, parts, n_windows,
                                                                  p.d_C + 2ll * woff * 64 * 64, p.d_status); break;
    default: return DH_ERR_UNSUPPORTED_SIZE;
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

// FP64 reduction of the covariance partials of windows [woff, woff + n_windows).
dh_status launch_reduce(Plan &p, int n_windows, int parts, int woff, cudaStream_t s) {
  switch (p.T) {
    case 16: return launch_reduce_t<16>(p, n_windows, parts, woff, s);
    case 32: return launch_reduce_t<32>(p, n_windows, parts, woff, s);
    case 64: return launch_reduce_t<64>(p, n_windows, parts, woff, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

// Eq. 5 + ordering + operand build for windows [woff, woff + n_windows); eig_user (if not
// NULL) already points at window woff's eigenvalues.
dh_status launch_jacobi(Plan &p, int n_windows, int k0, int k1, int Npad, double *eig_user, int woff,
                        cudaStream_t s, const SpanLayout *span) {
  switch (p.T) {
    case 16: return launch_jacobi_t<16>(p, n_windows, k0, k1, Npad, eig_user, woff, s, span);
    case 32: return launch_jacobi_t<32>(p, n_windows, k0, k1, Npad, eig_user, woff, s, span);
    case 64: return launch_jacobi_t<64>(p, n_windows, k0, k1, Npad, eig_user, woff, s, span);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace dh
