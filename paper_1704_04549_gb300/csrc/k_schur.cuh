// Real Schur form of a small dense matrix by one warp (Householder Hessenberg
// reduction, Francis double-shift QR with deflation from the bottom), shared by the
// factor build of the scalar blocks and of the full multi-component blocks.
#pragma once
#include "tpp_internal.cuh"

namespace tpp {
namespace {

constexpr double kEps = 2.220446049250313e-16;
// deflation threshold of the Francis iterations after 20 max(n, 8) steps without full
// convergence: sqrt(eps).  Clusters of nearly defective eigenvalues (e.g. the density
// blocks of the Euler systems, whose factors are a diagonal plus rank-one face terms)
// stall with subdiagonals near 1e-9; accepting them perturbs C by at most sqrt(eps) |C|.
constexpr double kRelax = 1.4901161193847656e-08;


__host__ __device__ __forceinline__ int ld_of(int n) { return (n & 1) ? n : n + 1; }

// ---- warp-level Householder helpers for the real Schur form --------------
// All lanes compute the same scalars from shared memory (uniform control).
__device__ void house_vec(const double* x, int len, double* v) {
  double nrm2 = 0.0;
  for (int i = 0; i < len; ++i) nrm2 += x[i] * x[i];
  for (int i = 0; i < len; ++i) v[i] = x[i];
  if (nrm2 == 0.0) {
    for (int i = 0; i < len; ++i) v[i] = 0.0;
    return;
  }
  const double nrm = sqrt(nrm2);
  v[0] += copysign(nrm, x[0]);
  const double inv = rsqrt(2.0 * nrm * (nrm + fabs(x[0])));   // ||v||^2 = 2 nrm (nrm + |x0|)
  for (int i = 0; i < len; ++i) v[i] *= inv;
}

// Real Schur form of H (n x n, column-major, leading dimension ld) in place,
// accumulating Q (initialised here).  Returns false when the Francis
// iteration exceeds its cap.  Executed by one full warp.
__device__ bool warp_real_schur(double* H, double* Q, int n, int ld, double* vb, bool* relaxed) {
  const int lane = threadIdx.x & 31;
  for (int r = lane; r < n; r += 32)
    for (int c = 0; c < n; ++c) Q[r + ld * c] = (r == c) ? 1.0 : 0.0;
  __syncwarp();
  // Householder reduction to upper Hessenberg form
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    double part = 0.0;
    for (int i = 1 + lane; i < L; i += 32) {
      const double xv = H[(k + 1 + i) + ld * k];
      part += xv * xv;
    }
    const double tail = warp_sum(part);
    if (tail == 0.0) continue;          // column already reduced
    const double alpha = H[(k + 1) + ld * k];
    const double nrm = sqrt(alpha * alpha + tail);
    const double v0 = alpha + copysign(nrm, alpha);
    const double inv = 1.0 / sqrt(v0 * v0 + tail);
    for (int i = lane; i < L; i += 32) vb[i] = (i == 0 ? v0 : H[(k + 1 + i) + ld * k]) * inv;
    __syncwarp();
    for (int c = k + lane; c < n; c += 32) {        // left: rows k+1.., columns k..
      double d = 0.0;
      for (int i = 0; i < L; ++i) d += vb[i] * H[(k + 1 + i) + ld * c];
      d *= 2.0;
      for (int i = 0; i < L; ++i) H[(k + 1 + i) + ld * c] -= d * vb[i];
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {            // right: columns k+1..
      double d = 0.0, dq = 0.0;
      for (int i = 0; i < L; ++i) {
        d += H[r + ld * (k + 1 + i)] * vb[i];
        dq += Q[r + ld * (k + 1 + i)] * vb[i];
      }
      d *= 2.0;
      dq *= 2.0;
      for (int i = 0; i < L; ++i) {
        H[r + ld * (k + 1 + i)] -= d * vb[i];
        Q[r + ld * (k + 1 + i)] -= dq * vb[i];
      }
    }
    __syncwarp();
    for (int i = 2 + lane; i < L + 1; i += 32) H[(k + i) + ld * k] = 0.0;
    __syncwarp();
  }
  double amax = 0.0;
  for (int c = lane; c < n; c += 32)
    for (int r = 0; r < n; ++r) amax = fmax(amax, fabs(H[r + ld * c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (amax == 0.0) return true;
  // Francis double-shift QR with deflation from the bottom
  int hi = n - 1, its = 0, total = 0;
  const int maxit = 40 * (n > 8 ? n : 8), relax = 20 * (n > 8 ? n : 8);
  while (hi > 0) {
    const double tol = (total > relax) ? kRelax : kEps;
    if (total > relax) *relaxed = true;
    int l = hi;
    while (l > 0) {
      double sc = fabs(H[(l - 1) + ld * (l - 1)]) + fabs(H[l + ld * l]);
      if (sc == 0.0) sc = amax;
      if (fabs(H[l + ld * (l - 1)]) <= tol * sc) break;
      --l;
    }
    __syncwarp();
    if (l > 0) {
      if (lane == 0) H[l + ld * (l - 1)] = 0.0;
      __syncwarp();
    }
    if (l == hi) { --hi; its = 0; continue; }
    if (l == hi - 1) { hi -= 2; its = 0; continue; }
    ++its;
    if (++total > maxit) return false;
    double s, t;
    if (its % 10 == 0) {
      // exceptional shift: the complex pair mu +- i sqrt(0.4375) w, w the size of the
      // last two subdiagonals, mu = H[hi][hi] + 0.75 w (a real double shift at mu stalls
      // on nearly defective eigenvalue clusters)
      const double w = fabs(H[hi + ld * (hi - 1)]) + fabs(H[(hi - 1) + ld * (hi - 2)]);
      const double mu = H[hi + ld * hi] + 0.75 * w;
      s = 2.0 * mu;
      t = mu * mu + 0.4375 * w * w;
    } else {                 // eigenvalues of the trailing 2 x 2 block
      const double a = H[(hi - 1) + ld * (hi - 1)], b = H[(hi - 1) + ld * hi];
      const double c = H[hi + ld * (hi - 1)], d = H[hi + ld * hi];
      s = a + d;
      t = a * d - b * c;
    }
    const double h00 = H[l + ld * l], h01 = H[l + ld * (l + 1)];
    const double h10 = H[(l + 1) + ld * l], h11 = H[(l + 1) + ld * (l + 1)];
    const double h21 = H[(l + 2) + ld * (l + 1)];
    double xv[3] = {h00 * h00 + h01 * h10 - s * h00 + t, h10 * (h00 + h11 - s), h10 * h21};
    double v[3];
    for (int k = l; k <= hi - 2; ++k) {
      house_vec(xv, 3, v);
      const int q = (k - 1 > l) ? k - 1 : l;
      __syncwarp();
      for (int c = q + lane; c < n; c += 32) {
        double* col = H + ld * c;
        const double d = 2.0 * (v[0] * col[k] + v[1] * col[k + 1] + v[2] * col[k + 2]);
        col[k] -= d * v[0];
        col[k + 1] -= d * v[1];
        col[k + 2] -= d * v[2];
      }
      __syncwarp();
      const int rmax = (k + 3 < hi) ? k + 3 : hi;
      for (int r = lane; r < n; r += 32) {
        if (r <= rmax) {
          const double d = 2.0 * (H[r + ld * k] * v[0] + H[r + ld * (k + 1)] * v[1] +
                                  H[r + ld * (k + 2)] * v[2]);
          H[r + ld * k] -= d * v[0];
          H[r + ld * (k + 1)] -= d * v[1];
          H[r + ld * (k + 2)] -= d * v[2];
        }
        const double dq = 2.0 * (Q[r + ld * k] * v[0] + Q[r + ld * (k + 1)] * v[1] +
                                 Q[r + ld * (k + 2)] * v[2]);
        Q[r + ld * k] -= dq * v[0];
        Q[r + ld * (k + 1)] -= dq * v[1];
        Q[r + ld * (k + 2)] -= dq * v[2];
      }
      __syncwarp();
      if (k > l && lane == 0) {
        H[(k + 1) + ld * (k - 1)] = 0.0;
        H[(k + 2) + ld * (k - 1)] = 0.0;
      }
      __syncwarp();
      xv[0] = H[(k + 1) + ld * k];
      xv[1] = H[(k + 2) + ld * k];
      xv[2] = (k < hi - 2) ? H[(k + 3) + ld * k] : 0.0;
    }
    house_vec(xv, 2, v);
    __syncwarp();
    for (int c = (hi - 2) + lane; c < n; c += 32) {
      double* col = H + ld * c;
      const double d = 2.0 * (v[0] * col[hi - 1] + v[1] * col[hi]);
      col[hi - 1] -= d * v[0];
      col[hi] -= d * v[1];
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {
      if (r <= hi) {
        const double d = 2.0 * (H[r + ld * (hi - 1)] * v[0] + H[r + ld * hi] * v[1]);
        H[r + ld * (hi - 1)] -= d * v[0];
        H[r + ld * hi] -= d * v[1];
      }
      const double dq = 2.0 * (Q[r + ld * (hi - 1)] * v[0] + Q[r + ld * hi] * v[1]);
      Q[r + ld * (hi - 1)] -= dq * v[0];
      Q[r + ld * hi] -= dq * v[1];
    }
    __syncwarp();
    if (lane == 0) H[hi + ld * (hi - 2)] = 0.0;
    __syncwarp();
  }
  return true;
}

}  // namespace
}  // namespace tpp
