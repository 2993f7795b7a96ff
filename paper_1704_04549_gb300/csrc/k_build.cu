// Per-element formation of the Kronecker preconditioner (Alg. 2d-form).
//
// One CTA per element:
//  1. coefficients of the rearranged block A~ = Q M Q^T (see k_struct_qr),
//  2. Golub-Kahan-Lanczos bidiagonalisation of M with full
//     reorthogonalisation (Alg. lanczos; Sec. 4.1.1 "full orthogonalization"),
//  3. top-2 singular triplets of the bidiagonal matrix: bisection on the
//     Golub-Kahan tridiagonal [[0, B], [B^T, 0]] (eigenvalues +-sigma) and
//     inverse iteration for the vectors; Ritz vectors back in A~ space,
//  4. A_k = sqrt(s_k) mat(u_k), B_k = sqrt(s_k) mat(v_k)  (column-major vec),
//  5. LU (Gauss-Jordan, partial pivoting) inverses of A_2 and B_1,
//     C_1 = A_2^-1 A_1, C_2 = B_1^-1 B_2 (Sec. 4.2),
//  6. real Schur forms C_i = Q_i T_i Q_i^T by Householder Hessenberg reduction
//     and Francis double-shift QR (one warp per matrix), Eq. quad-triang,
//  7. S_A = Q_1^T A_2^-1, S_B = Q_2^T B_1^-1 stored with Q_1, Q_2, T_1, T_2.
#include "tpp_internal.cuh"

namespace tpp {

namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr int kBuildThreads = 256;

struct BuildOut {
  double *sigma, *A1, *B1, *A2, *B2, *SA, *SB, *Q1, *Q2, *T1, *T2, *cond;
  int32_t* flags;
  uint32_t* masks;
  DevStatus* st;
};

__device__ __forceinline__ int ld_of(int n) { return (n & 1) ? n : n + 1; }

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
  double vn2 = 0.0;
  for (int i = 0; i < len; ++i) vn2 += v[i] * v[i];
  const double inv = 1.0 / sqrt(vn2);
  for (int i = 0; i < len; ++i) v[i] *= inv;
}

// Real Schur form of H (n x n, column-major, leading dimension ld) in place,
// accumulating Q (initialised here).  Returns false when the Francis
// iteration exceeds its cap.  Executed by one full warp.
__device__ bool warp_real_schur(double* H, double* Q, int n, int ld, double* vb) {
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
  const int maxit = 40 * (n > 8 ? n : 8);
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double sc = fabs(H[(l - 1) + ld * (l - 1)]) + fabs(H[l + ld * l]);
      if (sc == 0.0) sc = amax;
      if (fabs(H[l + ld * (l - 1)]) <= kEps * sc) break;
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
    if (its % 10 == 0) {     // exceptional shift: double real shift mu
      const double mu = H[hi + ld * hi] +
                        0.75 * (fabs(H[hi + ld * (hi - 1)]) + fabs(H[(hi - 1) + ld * (hi - 2)]));
      s = 2.0 * mu;
      t = mu * mu;
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

// ---- block / warp helpers --------------------------------------------------
// Sum of squares of v[0..len) computed by warp 0 and broadcast through *slot.
// FP64 warp instructions cost the full pipe width whatever their lane mask on
// this GPU, so short reductions run on one warp instead of the whole block.
__device__ double norm2_w0(const double* v, int len, double* slot) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int t = threadIdx.x; t < len; t += 32) s += v[t] * v[t];
    s = warp_sum(s);
    if (threadIdx.x == 0) *slot = s;
  }
  __syncthreads();
  return *slot;
}

__device__ double sum_w0(const double* v, int len, double* slot) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int t = threadIdx.x; t < len; t += 32) s += v[t];
    s = warp_sum(s);
    if (threadIdx.x == 0) *slot = s;
  }
  __syncthreads();
  return *slot;
}

// Reorthogonalise p (length r) against the first k vectors of B (vector-major,
// B[i*r + t]) twice: one warp per coefficient, then one thread per entry.
__device__ void reorth(double* p, const double* B, int k, int r, double* cf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pass = 0; pass < 2; ++pass) {
    __syncthreads();
    for (int i = wid; i < k; i += nw) {
      double s = 0.0;
      for (int t = lane; t < r; t += 32) s += B[i * r + t] * p[t];
      s = warp_sum(s);
      if (lane == 0) cf[i] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r; t += blockDim.x) {
      double s = p[t];
      for (int i = 0; i < k; ++i) s -= cf[i] * B[i * r + t];
      p[t] = s;
    }
  }
  __syncthreads();
}

// ---- Golub-Kahan tridiagonal T (zero diagonal, off-diagonal e, size m) ------
// Number of eigenvalues of T below x by the sign changes of the leading
// principal minors of T - x I (Sturm sequence): D_0 = 1, D_1 = -x,
// D_k = -x D_{k-1} - e_{k-2}^2 D_{k-2}.  e2 holds e^2 of the tridiagonal
// scaled to spectral radius <= 1, so no division is needed; an occasional
// rescale keeps D in range.
__device__ int sturm_count_df(const double* e2, int m, double x) {
  double d0 = 1.0, d1 = -x;
  int cnt = (d1 < 0.0) ? 1 : 0;
  bool neg_prev = d1 < 0.0;
  for (int k = 2; k <= m; ++k) {
    double d2 = fma(-x, d1, -e2[k - 2] * d0);
    bool neg = d2 < 0.0;
    if (d2 == 0.0) neg = !neg_prev;              // a zero minor counts as a sign change
    cnt += (neg != neg_prev) ? 1 : 0;
    neg_prev = neg;
    d0 = d1;
    d1 = d2;
    if ((k & 31) == 0 && fabs(d1) < 1e-200 && fabs(d0) < 1e-200) {
      d0 *= 1e200;
      d1 *= 1e200;
    }
  }
  return cnt;
}

// Inverse iteration on T - lam I (Gaussian elimination with partial pivoting,
// pivots inverted once); z in/out, work arrays of length m each.
__device__ void inverse_iteration(const double* e, int m, double lam, double* z, double* d,
                                  double* du, double* du2, double* dl, int* piv, double tiny) {
  for (int i = 0; i < m; ++i) {
    d[i] = -lam;
    du[i] = (i + 1 < m) ? e[i] : 0.0;
    dl[i] = (i + 1 < m) ? e[i] : 0.0;
    du2[i] = 0.0;
    piv[i] = 0;
  }
  for (int i = 0; i + 1 < m; ++i) {
    if (fabs(d[i]) >= fabs(dl[i])) {
      if (d[i] == 0.0) d[i] = tiny;
      const double f = dl[i] / d[i];
      dl[i] = f;
      d[i + 1] -= f * du[i];
    } else {       // exchange rows i and i+1
      const double f = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = f;
      const double tmp = du[i];
      du[i] = d[i + 1];
      d[i + 1] = tmp - f * d[i + 1];
      if (i + 2 < m) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
      piv[i] = 1;
    }
  }
  if (d[m - 1] == 0.0) d[m - 1] = tiny;
  for (int i = 0; i < m; ++i) d[i] = 1.0 / d[i];     // reciprocal pivots
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i + 1 < m; ++i) {     // L solve
      if (piv[i]) {
        const double t = z[i];
        z[i] = z[i + 1];
        z[i + 1] = t;
      }
      z[i + 1] -= dl[i] * z[i];
    }
    for (int i = m - 1; i >= 0; --i) {    // U solve
      double s = z[i];
      if (i + 1 < m) s -= du[i] * z[i + 1];
      if (i + 2 < m) s -= du2[i] * z[i + 2];
      z[i] = s * d[i];
    }
    double nr = 0.0;
    for (int i = 0; i < m; ++i) nr += z[i] * z[i];
    nr = 1.0 / sqrt(nr);
    for (int i = 0; i < m; ++i) z[i] *= nr;
  }
}

// Gauss-Jordan inverses of two n x n matrices at once (partial pivoting).
// aug[m] is n x 2n column-major (ld n): left block the matrix, right identity.
// Returns per-matrix singular flags in sing[2].
__device__ void gauss_jordan2(double* aug0, double* aug1, int n, int* pivrow, double* fac,
                              int* sing) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < n; ++k) {
    if (tid < 64) {                 // warp 0: matrix 0, warp 1: matrix 1 (lanes over rows)
      const int mIdx = tid >> 5, lane = tid & 31;
      const double* a = mIdx ? aug1 : aug0;
      double best = -1.0;
      int p = k;
      for (int i = k + lane; i < n; i += 32) {
        const double v = fabs(a[i + n * k]);
        if (v > best) { best = v; p = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (lane == 0) {
        pivrow[mIdx] = p;
        if (best == 0.0) sing[mIdx] = 1;
      }
    }
    __syncthreads();
    for (int q = tid; q < 2 * 2 * n; q += nt) {     // row swap
      const int mIdx = q / (2 * n), c = q % (2 * n);
      double* a = mIdx ? aug1 : aug0;
      const int p = pivrow[mIdx];
      if (p != k) {
        const double t = a[k + n * c];
        a[k + n * c] = a[p + n * c];
        a[p + n * c] = t;
      }
    }
    __syncthreads();
    for (int q = tid; q < 2 * n; q += nt) {         // multipliers (column k)
      const int mIdx = q / n, i = q % n;
      double* a = mIdx ? aug1 : aug0;
      const double piv = a[k + n * k];
      fac[mIdx * n + i] = (i == k) ? 0.0 : ((piv != 0.0) ? a[i + n * k] / piv : 0.0);
      if (i == k) fac[2 * n + mIdx] = (piv != 0.0) ? 1.0 / piv : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < 2 * n * 2 * n; q += nt) {   // eliminate + scale pivot row
      const int mIdx = q / (2 * n * n), rem = q % (2 * n * n);
      const int c = rem / n, i = rem % n;
      if (c < k) continue;
      double* a = mIdx ? aug1 : aug0;
      if (i == k) continue;
      a[i + n * c] -= fac[mIdx * n + i] * a[k + n * c];
    }
    __syncthreads();
    for (int q = tid; q < 2 * 2 * n; q += nt) {
      const int mIdx = q / (2 * n), c = q % (2 * n);
      if (c < k) continue;
      double* a = mIdx ? aug1 : aug0;
      a[k + n * c] *= fac[2 * n + mIdx];
    }
    __syncthreads();
  }
}

// 1-norm (max column sum) of an n x n column-major matrix by one warp.
__device__ double norm1_warp(const double* A, int n) {
  const int lane = threadIdx.x & 31;
  double best = 0.0;
  for (int c = lane; c < n; c += 32) {
    double sv = 0.0;
    for (int r = 0; r < n; ++r) sv += fabs(A[r + n * c]);
    best = fmax(best, sv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  return best;
}

__device__ void atomic_max_double(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
__device__ void atomic_min_double(double* addr, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace

// Shared-memory layout of k_build_2d (offsets in doubles).
struct BuildSmem {
  size_t cxs, cys, zds, rzs, big, vec, ints, total_bytes;
};

__host__ __device__ inline BuildSmem build_smem_layout(int n, int rz) {
  const int nc = n + 3, r = n + rz, nn = n * n;
  const int ld = (n & 1) ? n : n + 1;
  BuildSmem L;
  L.cxs = 0;
  L.cys = L.cxs + (size_t)nc * n;
  L.zds = L.cys + (size_t)nc * n;
  L.rzs = L.zds + (size_t)n * nc;
  L.big = L.rzs + (size_t)rz * nc;
  size_t big = (size_t)3 * r * r;
  const size_t need2 = (size_t)8 * nn + (size_t)4 * n * ld + 2 * n + 2 + 64;
  if (need2 > big) big = need2;
  L.vec = L.big + big;
  const size_t nvec = (size_t)16 * r + 1 + 16 + (size_t)16 * r;
  L.ints = L.vec + nvec;
  L.total_bytes = L.ints * sizeof(double) + (size_t)(4 * r + 8) * sizeof(int);
  return L;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBuildThreads)
k_build_2d(const Tables* T, int n, int rz, int nx, int ny, double h,
           const double* __restrict__ cx, const double* __restrict__ cy,
           const double* __restrict__ sx, const double* __restrict__ sy,
           const double* __restrict__ Zd, const double* __restrict__ Rz,
           const double* __restrict__ Qo, BuildOut out) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nn = n * n, nc = n + 3, r = n + rz, Ro = nn - n;
  const int64_t e = blockIdx.x;
  const int ex = (int)(e % nx), ey = (int)(e / nx);
  const int64_t eR = ey * (int64_t)nx + (ex + 1) % nx;
  const int64_t eT = ((ey + 1) % ny) * (int64_t)nx + ex;

  const BuildSmem L = build_smem_layout(n, rz);
  double* Cxs = sm + L.cxs;            // nc x n   Cx[c][j]
  double* Cys = sm + L.cys;            // nc x n   Cy[c][i]
  double* Zds = sm + L.zds;            // n x nc
  double* Rzs = sm + L.rzs;            // rz x nc
  double* big = sm + L.big;            // M (r*r), U (r*r), V (r*r); later n x n work
  double* Mm = big;
  double* U = Mm + r * r;
  double* V = U + r * r;
  double* pv = sm + L.vec;             // r
  double* cf = pv + r;                 // r
  double* al = cf + r;                 // r
  double* be = al + r;                 // r + 1
  double* ee = be + r + 1;             // 2r
  double* z1 = ee + 2 * r;             // 2r
  double* z2 = z1 + 2 * r;             // 2r
  double* e2s = z2 + 2 * r;            // 2r (squared scaled off-diagonal)
  double* mu1 = e2s + 2 * r;           // r  (Ritz vectors in M space)
  double* mv1 = mu1 + r;
  double* mu2 = mv1 + r;
  double* mv2 = mu2 + r;
  double* red = mv2 + r;               // 8
  double* scal = red + 8;              // 8 scalars
  double* tw = scal + 8;               // 2 x (4 * 2r) tridiagonal work
  int* piv = reinterpret_cast<int*>(sm + L.ints);   // 2 x 2r ints
  int* ish = piv + 2 * 2 * r;          // 8 ints

  // ---- 1. coefficients (flux Jacobians of the element, Sec. 3.4.1)
  const int64_t base = e * nn;
  for (int q = tid; q < nn; q += nt) {
    const int a = q % n, b = q / n;
    Cxs[a * n + b] = cx[base + q];      // Cx[c = x node][j]
    Cys[b * n + a] = cy[base + q];      // Cy[c = y node][i]
  }
  if (tid < n) {
    const int j = tid;
    Cxs[n * n + j] = fmax(sx[eR * n + j], 0.0);
    Cxs[(n + 1) * n + j] = fmax(-sx[e * n + j], 0.0);
    Cxs[(n + 2) * n + j] = h * h * T->w[j];
    Cys[n * n + j] = fmax(sy[eT * n + j], 0.0);
    Cys[(n + 1) * n + j] = fmax(-sy[e * n + j], 0.0);
    Cys[(n + 2) * n + j] = 0.0;
  }
  for (int q = tid; q < n * nc; q += nt) Zds[q] = Zd[q];
  for (int q = tid; q < rz * nc; q += nt) Rzs[q] = Rz[q];
  if (tid < 8) ish[tid] = 0;
  __syncthreads();

  // ---- 2. core matrix M (r x r, row-major)
  double fro = 0.0;
  for (int q = tid; q < r * r; q += nt) {
    const int p = q / r, c2 = q % r;
    double s = 0.0;
    if (p < n && c2 < n) {
      for (int c = 0; c < nc; ++c) s += Cxs[c * n + p] * Zds[c2 * nc + c] + Zds[p * nc + c] * Cys[c * n + c2];
    } else if (p < n) {
      const int t = c2 - n;
      for (int c = 0; c < nc; ++c) s += Cxs[c * n + p] * Rzs[t * nc + c];
    } else if (c2 < n) {
      const int t = p - n;
      for (int c = 0; c < nc; ++c) s += Rzs[t * nc + c] * Cys[c * n + c2];
    }
    Mm[q] = s;
    fro += s * s;
  }
  fro = sqrt(block_sum(fro, red));
  const double tol = 1e-12 * fro;

  // ---- 3. Golub-Kahan-Lanczos with full reorthogonalisation (Alg. lanczos)
  // Run J0 = min(r, 24) steps, take the top-2 Ritz triplets of the bidiagonal
  // and accept them when both residuals beta_J |u'_J| are below 1e-14 sigma_1;
  // otherwise continue to the full size r (a complete orthogonal reduction).
  {
    for (int t = tid; t < r; t += nt) V[t] = splitmix_unit(1, t);
    const double nv = sqrt(norm2_w0(V, r, &scal[3]));
    for (int t = tid; t < r; t += nt) V[t] /= nv;
    if (tid == 0) be[0] = 0.0;
    __syncthreads();
  }
  int J = (r < 24) ? r : 24;
  int jdone = 0;
  const int lane = tid & 31;
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = jdone; j < J; ++j) {
      // p = M v_j - beta_j u_{j-1}
      for (int t = tid; t < r; t += nt) {
        double sacc = 0.0;
        for (int q = 0; q < r; ++q) sacc += Mm[t * r + q] * V[j * r + q];
        if (j > 0) sacc -= be[j] * U[(j - 1) * r + t];
        pv[t] = sacc;
      }
      reorth(pv, U, j, r, cf);
      double a = sqrt(norm2_w0(pv, r, &scal[3]));
      if (a <= tol) {       // invariant subspace: continue with a fresh direction
        for (int t = tid; t < r; t += nt) pv[t] = splitmix_unit(1000 + j, t);
        reorth(pv, U, j, r, cf);
        const double nrm = sqrt(norm2_w0(pv, r, &scal[3]));
        for (int t = tid; t < r; t += nt) U[j * r + t] = pv[t] / nrm;
        a = 0.0;
      } else {
        const double ia = 1.0 / a;
        for (int t = tid; t < r; t += nt) U[j * r + t] = pv[t] * ia;
      }
      if (tid == 0) al[j] = a;
      __syncthreads();
      if (j + 1 < r) {
        // q = M^T u_j - alpha_j v_j
        for (int t = tid; t < r; t += nt) {
          double sacc = 0.0;
          for (int q = 0; q < r; ++q) sacc += Mm[q * r + t] * U[j * r + q];
          pv[t] = sacc - a * V[j * r + t];
        }
        reorth(pv, V, j + 1, r, cf);
        double b = sqrt(norm2_w0(pv, r, &scal[3]));
        if (b <= tol) {
          for (int t = tid; t < r; t += nt) pv[t] = splitmix_unit(2000 + j, t);
          reorth(pv, V, j + 1, r, cf);
          const double nrm = sqrt(norm2_w0(pv, r, &scal[3]));
          for (int t = tid; t < r; t += nt) V[(j + 1) * r + t] = pv[t] / nrm;
          b = 0.0;
        } else {
          const double ib = 1.0 / b;
          for (int t = tid; t < r; t += nt) V[(j + 1) * r + t] = pv[t] * ib;
        }
        if (tid == 0) be[j + 1] = b;
        __syncthreads();
      }
    }
    jdone = J;

    // ---- 4. top-2 singular values / vectors of the J x J bidiagonal matrix
    const int m = 2 * J;
    for (int t = tid; t < m - 1; t += nt) ee[t] = (t & 1) ? be[(t + 1) >> 1] : al[t >> 1];
    __syncthreads();
    if (tid < 32) {
      // Gershgorin bound of the spectrum, then e^2 of the scaled matrix
      double bnd = 0.0;
      for (int i = lane; i < m; i += 32) {
        const double sv = (i > 0 ? fabs(ee[i - 1]) : 0.0) + (i < m - 1 ? fabs(ee[i]) : 0.0);
        bnd = fmax(bnd, sv);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bnd = fmax(bnd, __shfl_xor_sync(0xffffffffu, bnd, o));
      if (bnd == 0.0) bnd = 1.0;
      const double ib = 1.0 / bnd;
      for (int i = lane; i < m - 1; i += 32) {
        const double es = ee[i] * ib;
        e2s[i] = es * es;
      }
      __syncwarp();
      // multisection: lanes 0-15 bracket the largest eigenvalue, 16-31 the second
      const int grp = lane >> 4, gl = lane & 15;
      const int idx = m - grp;
      double lo = 0.0, hi = 1.0 + 1e-12;
      for (int it = 0; it < 14; ++it) {
        const double x = lo + (hi - lo) * (double)(gl + 1) * (1.0 / 17.0);
        const int cnt = sturm_count_df(e2s, m, x);
        const unsigned ge = __ballot_sync(0xffffffffu, cnt >= idx);
        const unsigned mine = (ge >> (grp * 16)) & 0xffffu;
        const int f = mine ? (__ffs(mine) - 1) : 16;
        const double w = hi - lo;
        const double nlo = (f == 0) ? lo : lo + w * (double)f * (1.0 / 17.0);
        const double nhi = (f == 16) ? hi : lo + w * (double)(f + 1) * (1.0 / 17.0);
        lo = nlo;
        hi = nhi;
      }
      if (gl == 0) scal[grp] = (grp < J) ? 0.5 * (lo + hi) * bnd : 0.0;
      if (lane == 0) scal[4] = bnd;
      __syncwarp();
      // inverse iteration for both vectors in lockstep lanes 0 and 1
      if (lane < 2 && lane < J) {
        double* z = lane ? z2 : z1;
        for (int i = 0; i < m; ++i) z[i] = splitmix_unit(300 + lane, i);
        double* w0 = tw + lane * 4 * m;
        inverse_iteration(ee, m, scal[lane], z, w0, w0 + m, w0 + 2 * m, w0 + 3 * m, piv + lane * m,
                          kEps * bnd + 1e-300);
      }
      __syncwarp();
      if (lane == 0 && J >= 2) {          // z2 orthogonal to z1 (matters if sigma_1 ~ sigma_2)
        double dt = 0.0;
        for (int i = 0; i < m; ++i) dt += z1[i] * z2[i];
        double nr = 0.0;
        for (int i = 0; i < m; ++i) {
          z2[i] -= dt * z1[i];
          nr += z2[i] * z2[i];
        }
        nr = 1.0 / sqrt(nr);
        for (int i = 0; i < m; ++i) z2[i] *= nr;
      }
      if (lane == 0) {
        // residual of the Ritz triplets: beta_J |u'_{J-1}| with ||u'|| = 1/sqrt(2)
        const double bJ = (J < r) ? be[J] : 0.0;
        const double r1 = bJ * fabs(z1[m - 1]) * 1.4142135623730951;
        const double r2 = (J >= 2) ? bJ * fabs(z2[m - 1]) * 1.4142135623730951 : 0.0;
        scal[2] = (r1 <= 1e-14 * scal[0] && r2 <= 1e-14 * scal[0]) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    if (scal[2] != 0.0 || J == r) break;
    J = r;
  }
  const int nsv = (J >= 2) ? 2 : 1;
  // Ritz vectors: M v = sigma u with v = V v', u = U u'
  for (int k = 0; k < nsv; ++k) {
    const double* z = k ? z2 : z1;
    double* mu = k ? mu2 : mu1;
    double* mv = k ? mv2 : mv1;
    for (int sidx = tid; sidx < r; sidx += nt) {
      double a = 0.0, b = 0.0;
      for (int t = 0; t < J; ++t) {
        a += z[2 * t + 1] * U[t * r + sidx];
        b += z[2 * t] * V[t * r + sidx];
      }
      mu[sidx] = a;
      mv[sidx] = b;
    }
    const double pu = norm2_w0(mu, r, &scal[5]);
    const double pvv = norm2_w0(mv, r, &scal[6]);
    const double tr = sum_w0(mu, n, &scal[7]);
    const double sgn = (tr < 0.0) ? -1.0 : 1.0;     // gauge: trace(A_k) >= 0
    const double fu = sgn / sqrt(pu), fv = sgn / sqrt(pvv);
    for (int sidx = tid; sidx < r; sidx += nt) {
      mu[sidx] *= fu;
      mv[sidx] *= fv;
    }
    __syncthreads();
  }
  if (nsv == 1) {
    for (int sidx = tid; sidx < r; sidx += nt) { mu2[sidx] = 0.0; mv2[sidx] = 0.0; }
    if (tid == 0) scal[1] = 0.0;
    __syncthreads();
  }
  const double s1 = scal[0], s2 = scal[1];

  // ---- 5. factors A_k, B_k (n x n column-major): u = Q m_u, A_k = sqrt(s_k) mat(u)
  // Region "big" is free now; lay out the n x n work matrices there.
  const int ld = ld_of(n);
  double* fA1 = big;
  double* fB1 = fA1 + nn;
  double* fA2 = fB1 + nn;
  double* fB2 = fA2 + nn;
  double* aug0 = fB2 + nn;            // n x 2n
  double* aug1 = aug0 + 2 * nn;       // n x 2n
  double* H1 = aug1 + 2 * nn;         // n x ld
  double* H2 = H1 + n * ld;
  double* Qa = H2 + n * ld;
  double* Qb = Qa + n * ld;
  double* facv = Qb + n * ld;         // 2n + 2
  double* vb0 = facv + 2 * n + 2;     // 32
  double* vb1 = vb0 + 32;             // 32
  __syncthreads();
  {
    const double r1 = sqrt(s1), r2 = sqrt(s2);
    for (int q = tid; q < 4 * nn; q += nt) {
      const int which = q / nn, idx = q % nn;
      const int a = idx % n, b = idx / n;
      const double* mvec = (which == 0) ? mu1 : (which == 1) ? mv1 : (which == 2) ? mu2 : mv2;
      double val;
      if (a == b) {
        val = mvec[a];
      } else {
        const int o = b * (n - 1) + (a > b ? a - 1 : a);
        double s = 0.0;
        for (int t = 0; t < rz; ++t) s += Qo[(size_t)t * Ro + o] * mvec[n + t];
        val = s;
      }
      const double f = (which < 2) ? r1 : r2;
      double* dst = (which == 0) ? fA1 : (which == 1) ? fB1 : (which == 2) ? fA2 : fB2;
      dst[idx] = f * val;
    }
  }
  __syncthreads();
  for (int q = tid; q < nn; q += nt) {
    out.A1[base + q] = fA1[q];
    out.B1[base + q] = fB1[q];
    out.A2[base + q] = fA2[q];
    out.B2[base + q] = fB2[q];
  }
  if (tid == 0) {
    out.sigma[2 * e] = s1;
    out.sigma[2 * e + 1] = s2;
  }

  // ---- 6. factors to invert, inverses, C_1 and C_2
  // The paper inverts A_2 and B_1 (Sec. 4.2).  A rank-2 Kronecker sum is
  // unchanged by A_2 -> A_2 + alpha A_1, B_1 -> B_1 - alpha B_2, and A_2 alone
  // can be numerically singular while P is well conditioned, so alpha is taken
  // from a short list (alpha = t ||A_2|| / ||A_1||, t = 0 first) to minimise
  // cond_1(A_2 + alpha A_1) cond_1(B_1 - alpha B_2).  Rank-1 blocks invert A_1, B_1.
  const bool rank1 = !(s2 > 1e-14 * s1);
  const int mode = rank1 ? 2 : 0;
  const double tlist[7] = {0.0, 0.25, -0.25, 1.0, -1.0, 4.0, -4.0};
  double nA1 = 0.0, nA2 = 0.0;
  for (int q = tid; q < nn; q += nt) {
    nA1 += fA1[q] * fA1[q];
    nA2 += fA2[q] * fA2[q];
  }
  nA1 = block_sum(nA1, red);
  nA2 = block_sum(nA2, red);
  const double ascale = (nA1 > 0.0) ? sqrt(nA2 / nA1) : 0.0;
  double best = INFINITY, alpha = 0.0;
  int best_i = 0, last_i = -1;
  const int ncand = rank1 ? 1 : 7;
  for (int ci = 0; ci <= ncand; ++ci) {
    int use;
    if (ci < ncand) {
      use = ci;
    } else {                      // final pass: redo the best candidate if needed
      if (best_i == last_i) break;
      use = best_i;
    }
    const double al = rank1 ? 0.0 : tlist[use] * ascale;
    for (int q = tid; q < 2 * nn; q += nt) {
      const int c = q / n, rr = q % n;
      double va, vb;
      if (c < n) {
        const int idx = rr + n * c;
        va = rank1 ? fA1[idx] : fA2[idx] + al * fA1[idx];
        vb = rank1 ? fB1[idx] : fB1[idx] - al * fB2[idx];
      } else {
        va = vb = (rr == c - n) ? 1.0 : 0.0;
      }
      aug0[q] = va;
      aug1[q] = vb;
    }
    if (tid < 2) ish[2 + tid] = 0;
    __syncthreads();
    if (tid < 64) {     // 1-norms of the matrices before elimination (warp 0: A, warp 1: B)
      const double nv = norm1_warp((tid >> 5) ? aug1 : aug0, n);
      if ((tid & 31) == 0) scal[6 + (tid >> 5)] = nv;
    }
    __syncthreads();
    gauss_jordan2(aug0, aug1, n, ish, facv, ish + 2);
    if (tid < 64) {
      const double ni = norm1_warp((tid >> 5) ? aug1 + nn : aug0 + nn, n);
      if ((tid & 31) == 0) facv[2 * n + (tid >> 5)] = ni;   // scratch after elimination
    }
    __syncthreads();
    if (tid == 0) {
      double cp = scal[6] * facv[2 * n] * scal[7] * facv[2 * n + 1];
      if (ish[2] || ish[3] || !(cp < 1e300)) cp = INFINITY;
      scal[5] = cp;
    }
    __syncthreads();
    const double cp = scal[5];
    last_i = use;
    if (ci < ncand && cp < best) {
      best = cp;
      best_i = use;
      alpha = al;
    }
    if (ci < ncand && best <= 1e3) {
      best_i = use;
      break;
    }
    __syncthreads();
  }
  const double cond = best;
  const int sing = !(cond <= 1e14);
  const bool shifted = (alpha != 0.0);
  // C1 = LA^-1 A1 into H1, C2 = LB^-1 B2 into H2 (rank-1: C1 = 0, C2 = 0)
  {
    const double* LAi = aug0 + nn;
    const double* LBi = aug1 + nn;
    for (int q = tid; q < 2 * nn; q += nt) {
      const int which = q / nn, idx = q % nn;
      const int rr = idx % n, c = idx / n;
      double s = 0.0;
      if (mode != 2) {
        const double* Li = which ? LBi : LAi;
        const double* R = which ? fB2 : fA1;
        for (int k = 0; k < n; ++k) s += Li[rr + n * k] * R[k + n * c];
      }
      (which ? H2 : H1)[rr + ld * c] = s;
    }
  }
  __syncthreads();
  // ---- 7. real Schur forms (warp 0: C1, warp 1: C2)
  const int warp = tid >> 5;
  if (warp < 2) {
    const bool ok = warp_real_schur(warp ? H2 : H1, warp ? Qb : Qa, n, ld, warp ? vb1 : vb0);
    if ((tid & 31) == 0 && !ok) ish[4 + warp] = 1;
  }
  __syncthreads();
  const bool schur_fail = ish[4] || ish[5];
  if (mode == 2) {       // P = A1 (x) B1: T2 Y + Y T1^T = C with T1 = 0, T2 = I
    for (int q = tid; q < nn; q += nt) {
      const int rr = q % n, c = q / n;
      H2[rr + ld * c] = (rr == c) ? 1.0 : 0.0;
    }
    __syncthreads();
  }
  // ---- 8. S_A = Q1^T LA^-1, S_B = Q2^T LB^-1; outputs (column-major)
  {
    const double* LAi = aug0 + nn;
    const double* LBi = aug1 + nn;
    for (int q = tid; q < 2 * nn; q += nt) {
      const int which = q / nn, idx = q % nn;
      const int rr = idx % n, c = idx / n;
      const double* Qm = which ? Qb : Qa;
      const double* Li = which ? LBi : LAi;
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += Qm[k + ld * rr] * Li[k + n * c];
      (which ? out.SB : out.SA)[base + idx] = s;
      (which ? out.Q2 : out.Q1)[base + idx] = Qm[rr + ld * c];
      (which ? out.T2 : out.T1)[base + idx] = (which ? H2 : H1)[rr + ld * c];
    }
  }
  if (tid == 0) {
    uint32_t m1 = 0, m2 = 0;
    for (int i = 0; i + 1 < n; ++i) {
      if (H1[(i + 1) + ld * i] != 0.0) m1 |= 1u << i;
      if (H2[(i + 1) + ld * i] != 0.0) m2 |= 1u << i;
    }
    out.masks[2 * e] = m1;
    out.masks[2 * e + 1] = m2;
    int fl = 0;
    if (shifted) fl |= 1;
    if (mode == 2) fl |= 2;
    if (schur_fail) fl |= 4;
    if (sing) fl |= 8;
    out.flags[e] = fl;
    out.cond[e] = cond;
    if (shifted) atomicAdd(&out.st->build_shifted, 1);
    if (mode == 2) atomicAdd(&out.st->build_rank1, 1);
    if (schur_fail) atomicAdd(&out.st->build_schur_fail, 1);
    if (sing) atomicAdd(&out.st->build_singular, 1);
    if (cond < 1e300) atomic_max_double(&out.st->max_cond, cond);
    atomic_min_double(&out.st->min_sigma_ratio, (s1 > 0.0) ? s2 / s1 : 0.0);
  }
}

cudaError_t launch_build_2d(const tpp_ctx* c, cudaStream_t s) {
  const int n = c->n;
  const size_t smem = build_smem_layout(n, c->rz).total_bytes;
  cudaError_t err = cudaFuncSetAttribute(k_build_2d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  BuildOut o;
  o.sigma = c->p<double>(c->L.sigma);
  o.A1 = c->p<double>(c->L.fA1);
  o.B1 = c->p<double>(c->L.fB1);
  o.A2 = c->p<double>(c->L.fA2);
  o.B2 = c->p<double>(c->L.fB2);
  o.SA = c->p<double>(c->L.fSA);
  o.SB = c->p<double>(c->L.fSB);
  o.Q1 = c->p<double>(c->L.fQ1);
  o.Q2 = c->p<double>(c->L.fQ2);
  o.T1 = c->p<double>(c->L.fT1);
  o.T2 = c->p<double>(c->L.fT2);
  o.cond = c->p<double>(c->L.fSC);
  o.flags = c->p<int32_t>(c->L.flags);
  o.masks = c->p<uint32_t>(c->L.masks);
  o.st = c->p<DevStatus>(c->L.status);
  k_build_2d<<<(unsigned)c->E, kBuildThreads, smem, s>>>(
      c->p<Tables>(c->L.tables), n, c->rz, c->prob.nel[0], c->prob.nel[1], c->prob.h,
      c->p<double>(c->L.cx), c->p<double>(c->L.cy), c->p<double>(c->L.sx),
      c->p<double>(c->L.sy), c->p<double>(c->L.zd), c->p<double>(c->L.rz),
      c->p<double>(c->L.qo), o);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
