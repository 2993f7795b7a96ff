// Per-element formation of the Kronecker preconditioner (Alg. 2d-form):
//  1. coefficients of the rearranged block A~ = Q M Q^T (see k_struct_qr),
//  2. dense Householder bidiagonalisation of the small core M (the paper runs
//     Lanczos on A~, Sec. 4.1.1; the triplets are the same),
//  3. top-2 singular triplets of the bidiagonal matrix: bisection on the
//     Golub-Kahan tridiagonal [[0, B], [B^T, 0]] (eigenvalues +-sigma),
//     inverse iteration for the vectors, reflectors applied back,
//  4. A_k = sqrt(s_k) mat(u_k), B_k = sqrt(s_k) mat(v_k)  (column-major vec),
//  5. Gauss-Jordan inverses of the gauge-shifted pair A_2 + alpha A_1 and
//     B_1 - alpha B_2 (the paper's A_2, B_1 for alpha = 0), C_1 = L_A^-1 A_1,
//     C_2 = L_B^-1 B_2 (Sec. 4.2),
//  6. real Schur forms C_i = Q_i T_i Q_i^T by Householder Hessenberg reduction
//     and Francis double-shift QR, Eq. quad-triang (C_1 only in the one-sided
//     form, whose shifted systems C_2 + T_1[J, J] are then inverted),
//  7. S_A = Q_1^T L_A^-1 (and S_B = Q_2^T L_B^-1) stored with Q_1, T_1 (Q_2, T_2).
#include "tpp_internal.cuh"
#include "k_schur.cuh"

namespace tpp {

namespace {


// ---- two real Schur forms per warp (n <= 16), one per half-warp -----------
// The algorithm of warp_real_schur (Householder Hessenberg reduction, Francis
// double-shift sweeps with deflation from the bottom) run by each half-warp on
// its own matrix in lockstep: the bulge-chasing loop runs to the longer of the
// two active windows and a half whose matrix has converged idles.  Every FP64
// instruction then serves two matrices (on GB300 a warp FP64 instruction costs
// the pipe the same with 16 or 32 active lanes).  Deflation: the negligible
// subdiagonal entries of a half are found in parallel (one lane per position,
// a ballot) and the window update is integer work.
__device__ bool hw_real_schur(double* H, double* Q, int n, int ld, double* vb, bool empty,
                              bool* relaxed) {
  const int lane = threadIdx.x & 31, hl = lane & 15, hb = lane & 16;
  for (int c = 0; c < n; ++c)
    if (hl < n) Q[hl + ld * c] = (hl == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int k = 0; k + 2 < n; ++k) {                 // Hessenberg reduction (uniform)
    const int L = n - k - 1;
    const double xh = (1 + hl < L) ? H[(k + 1 + 1 + hl) + ld * k] : 0.0;
    double tail = xh * xh;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
    const double alpha = H[(k + 1) + ld * k];
    const double nrm = sqrt(alpha * alpha + tail);
    const double v0 = alpha + copysign(nrm, alpha);
    const double inv = (tail != 0.0) ? rsqrt(v0 * v0 + tail) : 0.0;   // tail = 0: identity
    if (hl < L) vb[hb + hl] = (hl == 0 ? v0 : H[(k + 1 + hl) + ld * k]) * inv;
    __syncwarp();
    const double* v = vb + hb;
    if (k + hl < n) {                               // left: rows k+1.., column k + hl
      const int c = k + hl;
      double d = 0.0;
      for (int i = 0; i < L; ++i) d += v[i] * H[(k + 1 + i) + ld * c];
      d *= 2.0;
      for (int i = 0; i < L; ++i) H[(k + 1 + i) + ld * c] -= d * v[i];
    }
    __syncwarp();
    if (hl < n) {                                   // right: columns k+1.., row hl
      const int r = hl;
      double d = 0.0, dq = 0.0;
      for (int i = 0; i < L; ++i) {
        d += H[r + ld * (k + 1 + i)] * v[i];
        dq += Q[r + ld * (k + 1 + i)] * v[i];
      }
      d *= 2.0;
      dq *= 2.0;
      for (int i = 0; i < L; ++i) {
        H[r + ld * (k + 1 + i)] -= d * v[i];
        Q[r + ld * (k + 1 + i)] -= dq * v[i];
      }
    }
    __syncwarp();
    if (inv != 0.0 && 2 + hl < L + 1) H[(k + 2 + hl) + ld * k] = 0.0;
    __syncwarp();
  }
  double amax = 0.0;
  for (int c = 0; c < n; ++c)
    if (hl < n) amax = fmax(amax, fabs(H[hl + ld * c]));
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  int hi = (empty || amax == 0.0) ? 0 : n - 1, its = 0, total = 0;
  bool fail = false;
  const int maxit = 40 * (n > 8 ? n : 8), relax = 20 * (n > 8 ? n : 8);
  while (true) {
    // negligible subdiagonal entries (position i = hl + 1: H[i][i-1])
    bool small = false;
    {
      const int i = hl + 1;
      if (total > relax) *relaxed = true;
      if (i < n && hi > 0) {
        double sc = fabs(H[(i - 1) + ld * (i - 1)]) + fabs(H[i + ld * i]);
        if (sc == 0.0) sc = amax;
        small = fabs(H[i + ld * (i - 1)]) <= ((total > relax) ? kRelax : kEps) * sc;
      }
    }
    const unsigned mine = (__ballot_sync(0xffffffffu, small) >> hb) & 0xffffu;
    __syncwarp();
    if (small && hl + 1 <= hi) H[(hl + 1) + ld * hl] = 0.0;
    int l = 0;
    while (hi > 0) {                                // deflation: integer work
      const unsigned mm = mine & ((hi >= 16) ? 0xffffu : ((1u << hi) - 1u));
      l = mm ? (32 - __clz(mm)) : 0;
      if (l == hi) { --hi; its = 0; continue; }
      if (l == hi - 1) { hi -= 2; its = 0; continue; }
      break;
    }
    bool go = hi > 0 && !fail;
    if (go) {
      ++its;
      if (++total > maxit) {
        fail = true;
        go = false;
      }
    }
    if (!__any_sync(0xffffffffu, go)) break;
    __syncwarp();
    // shifts (indices clamped for an idle half; its values are not used)
    const int h2 = go ? hi : 2, l2 = go ? l : 0;
    double sh, t;
    if (its % 10 == 0) {     // exceptional complex shift pair (as in k_schur_w)
      const double w = fabs(H[h2 + ld * (h2 - 1)]) + fabs(H[(h2 - 1) + ld * (h2 - 2)]);
      const double mu = H[h2 + ld * h2] + 0.75 * w;
      sh = 2.0 * mu;
      t = mu * mu + 0.4375 * w * w;
    } else {
      const double a = H[(h2 - 1) + ld * (h2 - 1)], b = H[(h2 - 1) + ld * h2];
      const double c = H[h2 + ld * (h2 - 1)], d = H[h2 + ld * h2];
      sh = a + d;
      t = a * d - b * c;
    }
    const double h00 = H[l2 + ld * l2], h01 = H[l2 + ld * (l2 + 1)];
    const double h10 = H[(l2 + 1) + ld * l2], h11 = H[(l2 + 1) + ld * (l2 + 1)];
    const double h21 = H[(l2 + 2) + ld * (l2 + 1)];
    double xv[3] = {h00 * h00 + h01 * h10 - sh * h00 + t, h10 * (h00 + h11 - sh), h10 * h21};
    double v[3];
    const int nst = go ? hi - 1 - l : 0;            // bulge steps k = l .. hi - 2
    const int nmax = max(nst, __shfl_xor_sync(0xffffffffu, nst, 16));
    for (int kk = 0; kk < nmax; ++kk) {
      const int k = l2 + kk;
      const bool a = kk < nst;
      house_vec(xv, 3, v);
      const int q = (k - 1 > l2) ? k - 1 : l2;
      if (a && q + hl < n) {
        double* col = H + ld * (q + hl);
        const double d = 2.0 * (v[0] * col[k] + v[1] * col[k + 1] + v[2] * col[k + 2]);
        col[k] -= d * v[0];
        col[k + 1] -= d * v[1];
        col[k + 2] -= d * v[2];
      }
      __syncwarp();
      if (a && hl < n) {
        const int r = hl;
        const int rmax = (k + 3 < hi) ? k + 3 : hi;
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
      if (a && k > l2 && hl == 0) {
        H[(k + 1) + ld * (k - 1)] = 0.0;
        H[(k + 2) + ld * (k - 1)] = 0.0;
      }
      __syncwarp();
      if (a) {                                      // a finished half keeps its last bulge
        xv[0] = H[(k + 1) + ld * k];
        xv[1] = H[(k + 2) + ld * k];
        xv[2] = (k < hi - 2) ? H[(k + 3) + ld * k] : 0.0;
      }
    }
    house_vec(xv, 2, v);
    if (go && (h2 - 2) + hl < n) {
      double* col = H + ld * ((h2 - 2) + hl);
      const double d = 2.0 * (v[0] * col[h2 - 1] + v[1] * col[h2]);
      col[h2 - 1] -= d * v[0];
      col[h2] -= d * v[1];
    }
    __syncwarp();
    if (go && hl < n) {
      const int r = hl;
      if (r <= h2) {
        const double d = 2.0 * (H[r + ld * (h2 - 1)] * v[0] + H[r + ld * h2] * v[1]);
        H[r + ld * (h2 - 1)] -= d * v[0];
        H[r + ld * h2] -= d * v[1];
      }
      const double dq = 2.0 * (Q[r + ld * (h2 - 1)] * v[0] + Q[r + ld * h2] * v[1]);
      Q[r + ld * (h2 - 1)] -= dq * v[0];
      Q[r + ld * h2] -= dq * v[1];
    }
    __syncwarp();
    if (go && hl == 0) H[h2 + ld * (h2 - 2)] = 0.0;
    __syncwarp();
  }
  return !fail;
}

// ---- Golub-Kahan tridiagonal T (zero diagonal, off-diagonal e, size m) ------
// Sturm counts: sturm_count_gk (k_ksvd_tri) counts the eigenvalues of T below x
// by the sign changes of the leading principal minors of T - x I: D_0 = 1,
// D_1 = -x, D_k = -x D_{k-1} - e_{k-2}^2 D_{k-2}, with e scaled to spectral
// radius <= 1 (no division) and an occasional rescale to keep D in range.

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

// ---------------------------------------------------------------------------
// Build pipeline (2D).  A warp-wide FP64 instruction costs the FP64 pipe the
// same (16 SM cycles) whatever its active lanes, so the work is laid out for
// full warps:
//   k_ksvd_w       warp per element: core M of the rearranged block
//                  (r = n + rz), dense Householder bidiagonalisation
//   k_ksvd_tri     thread per (element, k): sigma_k by bisection, its vector
//                  by inverse iteration on the Golub-Kahan tridiagonal
//   k_ksvd_vec     warp per element: reflectors back (four vectors in lane
//                  groups), factors A_k, B_k                           (a3, a4)
//   k_invert_r     n <= 16: gauge candidates ranked in FP32, the chosen pair
//                  inverted in FP64, both matrices in one warp (k_invert_w:
//                  n > 16, shared-memory Gauss-Jordan); C_1, C_2        (a5)
//   k_schur_w2     n <= 16: two real Schur forms per warp (k_schur_w: n > 16)
//   k_shift_inv_r  one-sided form, n <= 16: inverses of the shifted diagonal
//                  systems of every column block of T_1 (complex n x n for the
//                  2x2 blocks; k_shift_inv_fb the nearly defective ones;
//                  k_shift_inv_w: n > 16)
//   k_final_w      S_A = Q_1^T L_A^-1 (two-sided: also S_B = Q_2^T L_B^-1)

struct KsvdArgs {
  int n, rz;           // core size r = n + rz
  int64_t E;
  const double* kco;   // per block: Cx ((n+2) x n), Cy ((n+2) x n), Dg (n x n)
  const double *Zd, *Rz, *Qo;
  // over-integrated blocks (mu > n): the core of every element given explicitly
  // (Mcore [E][r x r] column-major), A~ = Qb M Qb^T with the dense orthonormal basis
  // Qb (column-major n^2 x r) and qtr[t] = trace of mat(Qb[:, t]); NULL otherwise
  const double *Mcore, *Qb, *qtr;
  double* scr;     // per element: the k_ksvd_w shared-memory image, tridiagonal work (16 r)
  int* iscr;       // per element: 4 r pivot flags
  double *sigma, *A1, *B1, *A2, *B2;
  DevStatus* st;
  const int32_t* mask;   // optional: only elements with mask[e] != 0 are decomposed
};

// shared-memory layout of one warp of k_ksvd_w (offsets in doubles): the core
// M (r x r, odd leading dimension against bank conflicts), the bidiagonal,
// the Golub-Kahan tridiagonal and its two eigenvectors, the singular vectors
// in M coordinates and the Householder scalars
struct KsvdSmem {
  int M, ldm, al, be, ee, e2s, z1, z2, mu1, mv1, mu2, mv2, tl, tr, scal, total;
};

__host__ __device__ inline KsvdSmem ksvd_smem(int n, int rz) {
  const int r = n + rz;
  KsvdSmem L;
  int o = 0;
  L.ldm = r | 1;
  L.M = o; o += r * L.ldm;
  L.al = o; o += r;
  L.be = o; o += r + 1;
  L.ee = o; o += 2 * r;
  L.e2s = o; o += 2 * r;
  L.z1 = o; o += 2 * r;
  L.z2 = o; o += 2 * r;
  L.mu1 = o; o += r;
  L.mv1 = o; o += r;
  L.mu2 = o; o += r;
  L.mv2 = o; o += r;
  L.tl = o; o += r;
  L.tr = o; o += r;
  L.scal = o; o += 8;
  L.total = (o + 1) & ~1;
  return L;
}

namespace {

// p (shared, length r) minus its projections on the first k rows of B
// (global, row i at B + i r), twice; coefficients 32 at a time, one per lane.
__device__ void warp_reorth(double* p, const double* B, int k, int r, double* cf) {
  const int lane = threadIdx.x & 31;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i0 = 0; i0 < k; i0 += 32) {
      const int i = i0 + lane;
      double sv = 0.0;
      if (i < k) {
        const double* bi = B + (size_t)i * r;
        for (int t = 0; t < r; ++t) sv += bi[t] * p[t];
      }
      cf[lane] = sv;
      __syncwarp();
      const int cnt = (k - i0 < 32) ? k - i0 : 32;
      for (int t = lane; t < r; t += 32) {
        double v = p[t];
        for (int q = 0; q < cnt; ++q) v -= cf[q] * B[(size_t)(i0 + q) * r + t];
        p[t] = v;
      }
      __syncwarp();
    }
  }
}

// Gauss-Jordan inverse of the n x n left half of a (n x 2n, column-major, ld n)
// with partial pivoting, by one warp (lanes over columns).  Returns true if a
// zero pivot was met.  fac: n scratch.
__device__ bool warp_gauss_jordan(double* a, int n, double* fac) {
  const int lane = threadIdx.x & 31;
  bool sing = false;
  for (int k = 0; k < n; ++k) {
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
    if (best == 0.0) sing = true;
    if (p != k)
      for (int c = lane; c < 2 * n; c += 32) {
        const double t = a[k + n * c];
        a[k + n * c] = a[p + n * c];
        a[p + n * c] = t;
      }
    __syncwarp();
    const double piv = a[k + n * k];
    const double ip = (piv != 0.0) ? 1.0 / piv : 0.0;
    for (int i = lane; i < n; i += 32) fac[i] = (i == k) ? 0.0 : a[i + n * k] * ip;
    __syncwarp();
    for (int c = k + lane; c < 2 * n; c += 32) {
      const double akc = a[k + n * c];
      for (int i = 0; i < n; ++i) a[i + n * c] -= fac[i] * akc;
      a[k + n * c] = akc * ip;
    }
    __syncwarp();
  }
  return sing;
}

// Gauss-Jordan inverse of an m x m matrix (m <= M <= 32) held by rows in
// registers: lane r < m holds row r in a[].  Pivot rows are chosen by largest
// magnitude (compared on the upper 32 bits of |a|, integer pipe) and never
// exchanged; rows are not normalised during the elimination (each step is one
// FMA per remaining entry for every row but the pivot row), so at the end row r
// of [A | I] reads [d_r e_{k_r} | d_r (row k_r of A^-1)].  On return b[] of lane
// r holds row k_r of A^-1 and the function returns k_r (-1 for lanes >= m).
// `sing` is set when a pivot is zero (its row of the inverse is then left 0).
// In-place Gauss-Jordan inverse of the m x m matrix whose row l sits in lane l's
// registers (m <= M <= 32), partial pivoting without row exchanges: at step k the
// pivot row p scales to (row_p / a_pk, with 1 / a_pk in column k) and every other
// row r takes row_r - f row_p (f = a_rk / a_pk, -f in column k).  On return lane r
// holds, in slot c, entry (kr, piv[c]) of the inverse, kr the step at which row r
// was the pivot (-1 for lanes >= m).  M FMAs per lane and step (the augmented
// [A | I] form needs up to 2M).  Pivot search on the magnitude bits (integer pipe).
__device__ __forceinline__ int mag_key(float v) { return __float_as_int(v) & 0x7fffffff; }
__device__ __forceinline__ int mag_key(double v) { return __double2hiint(v) & 0x7fffffff; }

// in-place Gauss-Jordan inverse of an m x m matrix with row l in lane l (T = double or
// float: the one-sided shifted inverses may be formed in FP32 for the FP32 apply)
template <int M, typename T = double>
__device__ __forceinline__ int warp_gj_inplace(T (&a)[M], int (&piv)[M], int m, bool& sing) {
  const int lane = threadIdx.x & 31;
  bool used = lane >= m;
  int kr = -1;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    piv[k] = 0;
    if (k < m) {
      const int key = used ? -1 : mag_key(a[k]);
      const int mx = __reduce_max_sync(0xffffffffu, key);
      unsigned bal = __ballot_sync(0xffffffffu, !used && key == mx);
      if (mx <= 0) {
        sing = true;
        bal = __ballot_sync(0xffffffffu, !used);
      }
      const int p = __ffs(bal) - 1;
      const T pv = __shfl_sync(0xffffffffu, a[k], p);
      const T ip = (pv != T(0)) ? T(1) / pv : T(0);
      const bool isp = (lane == p);
      const T f = a[k] * ip;
      const T s1 = isp ? ip : -f;
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if (c == k || c >= m) continue;
        const T v = __shfl_sync(0xffffffffu, a[c], p);
        a[c] = fma(s1, v, isp ? T(0) : a[c]);
      }
      a[k] = s1;
      if (isp) {
        used = true;
        kr = k;
      }
      piv[k] = p;
    }
  }
  return kr;
}

// Complex version for n <= 16: the n x n complex matrix Y0 = C_2 + mu I with row l's
// real part in lane l and imaginary part in lane l + 16; same in-place scheme.
template <typename T = double>
__device__ __forceinline__ int warp_gj_inplace_c(T (&a)[16], uint64_t& piv, int n, bool& sing) {
  const int lane = threadIdx.x & 31, row = lane & 15;
  const bool im = lane >= 16;
  bool used = row >= n;
  int kr = -1;
  piv = 0;                      // pivot row of step k in bits 4k..4k+3
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < n) {
      const T ak = a[k];
      const T ao = __shfl_xor_sync(0xffffffffu, ak, 16);
      const int key = used ? -1 : max(mag_key(ak), mag_key(ao));
      const int mx = __reduce_max_sync(0xffffffffu, key);
      unsigned bal = __ballot_sync(0xffffffffu, !used && !im && key == mx);
      if (mx <= 0) {
        sing = true;
        bal = __ballot_sync(0xffffffffu, !used && !im);
      }
      const int p = __ffs(bal) - 1;
      const T pr = __shfl_sync(0xffffffffu, ak, p);
      const T pi = __shfl_sync(0xffffffffu, ak, p + 16);
      const T den = pr * pr + pi * pi;
      const T iden = (den != T(0)) ? T(1) / den : T(0);
      const T ipr = pr * iden, ipi = -pi * iden;
      const T akr = im ? ao : ak, aki = im ? ak : ao;
      const T fr = akr * ipr - aki * ipi, fi = akr * ipi + aki * ipr;
      const bool isp = (row == p);
      // lane value of row_r - f row_p (re: b - fr vr + fi vi, im: b - fr vi - fi vr);
      // pivot row: ip row_p (re: ipr vr - ipi vi, im: ipr vi + ipi vr)
      const T s1 = isp ? ipr : -fr;
      const T s2 = isp ? (im ? ipi : -ipi) : (im ? -fi : fi);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (c == k || c >= n) continue;
        const T vr = __shfl_sync(0xffffffffu, a[c], p);
        const T vi = __shfl_sync(0xffffffffu, a[c], p + 16);
        a[c] = fma(s1, im ? vi : vr, fma(s2, im ? vr : vi, isp ? T(0) : a[c]));
      }
      a[k] = isp ? (im ? ipi : ipr) : (im ? -fi : -fr);
      if (isp) {
        used = true;
        kr = k;
      }
      piv |= (uint64_t)p << (4 * k);
    }
  }
  return kr;
}

}  // namespace

// The core M of the rearranged block, A~ = Q M Q^T (Q = [E | Qo]):
// M = [[Cx^T Zd^T + Zd Cy + Dg^T, Cx^T Rz^T], [Rz Cy, 0]], written column-major
// (leading dimension ld) by one warp.
__device__ void form_core(const double* Cx, const double* Cy, const double* Dg, const double* Zd,
                          const double* Rz, int n, int rz, double* Ms, int ld) {
  const int nc = n + 2, r = n + rz, lane = threadIdx.x & 31;
  for (int q = lane; q < r * r; q += 32) {
    const int i = q % r, j = q / r;
    double v = 0.0;
    if (i < n && j < n) {
      for (int c = 0; c < nc; ++c)
        v += __ldg(Cx + c * n + i) * __ldg(Zd + j * nc + c) +
             __ldg(Zd + i * nc + c) * __ldg(Cy + c * n + j);
      v += __ldg(Dg + j + n * i);
    } else if (i < n) {
      const int t = j - n;
      for (int c = 0; c < nc; ++c) v += __ldg(Cx + c * n + i) * __ldg(Rz + t * nc + c);
    } else if (j < n) {
      const int t = i - n;
      for (int c = 0; c < nc; ++c) v += __ldg(Rz + t * nc + c) * __ldg(Cy + c * n + j);
    }
    Ms[i + ld * j] = v;
  }
}

// ---- KSVD in three stages (one-thread scalar work is split out: on GB300 an
// FP64 warp instruction costs the pipe the same with 1 or 32 active lanes):
//  k_ksvd_w    warp per element: core M, Householder bidiagonalisation; the
//              warp's shared-memory image goes to the element's scratch,
//  k_ksvd_tri  thread per (element, k), k = 0, 1: k-th largest eigenvalue of
//              the Golub-Kahan tridiagonal (bisection on Sturm counts) and its
//              eigenvector (inverse iteration),
//  k_ksvd_vec  warp per element: singular vectors back in M coordinates
//              (reflectors last to first) and the factors A_k, B_k.
// Scratch per element (doubles): the image (ksvd_smem total) then 16 r of
// tridiagonal work; ksvd_scr_stride() of them.
__host__ __device__ inline size_t ksvd_scr_stride(int n, int rz) {
  return (size_t)ksvd_smem(n, rz).total + 16 * (size_t)(n + rz);
}

__global__ void __launch_bounds__(128) k_ksvd_w(KsvdArgs A) {
  extern __shared__ double smk[];
  const int n = A.n, rz = A.rz, nc = n + 2, r = n + rz, nn = n * n, Ro = nn - n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= A.E) return;                                  // whole warp leaves together
  const KsvdSmem L = ksvd_smem(n, rz);
  double* sm = smk + (size_t)warp * L.total;
  double* Ms = sm + L.M;
  const int ld = L.ldm;
  double *al = sm + L.al, *be = sm + L.be, *tl = sm + L.tl, *tr = sm + L.tr;
  double* Sg = A.scr + (size_t)e * ksvd_scr_stride(n, rz);
  const double* kc = A.kco + (size_t)e * (2 * nc * n + nn);
  const double *Cx = kc, *Cy = kc + nc * n, *Dg = kc + 2 * nc * n;

  if (A.mask && !A.mask[e]) return;                     // factors given (whole warp)
  if (A.Mcore) {
    const double* Mg = A.Mcore + (size_t)e * r * r;
    for (int q = lane; q < r * r; q += 32) Ms[(q % r) + ld * (q / r)] = Mg[q];
  } else {
    form_core(Cx, Cy, Dg, A.Zd, A.Rz, n, rz, Ms, ld);
  }
  __syncwarp();

  // ---- Householder bidiagonalisation M = U_h B V_h^T (B upper bidiagonal:
  // diagonal al[k], superdiagonal be[k + 1]); the reflector vectors stay in
  // M below the diagonal (left, unit first entry implied) and right of the
  // superdiagonal (right)
  for (int k = 0; k < r; ++k) {
    double* colk = Ms + ld * k;
    double sg = 0.0;
    for (int i = k + 1 + lane; i < r; i += 32) sg += colk[i] * colk[i];
    sg = warp_sum(sg);
    const double x0 = colk[k];
    double tau = 0.0, alpha = x0;
    if (sg > 0.0) {
      const double nx = sqrt(x0 * x0 + sg);
      alpha = (x0 > 0.0) ? -nx : nx;
      tau = (alpha - x0) / alpha;
      const double iv = 1.0 / (x0 - alpha);
      for (int i = k + 1 + lane; i < r; i += 32) colk[i] *= iv;
    }
    __syncwarp();
    if (tau != 0.0) {
      for (int j = k + 1 + lane; j < r; j += 32) {
        double* cj = Ms + ld * j;
        double sv = cj[k];
        for (int i = k + 1; i < r; ++i) sv += colk[i] * cj[i];
        sv *= tau;
        cj[k] -= sv;
        for (int i = k + 1; i < r; ++i) cj[i] -= sv * colk[i];
      }
    }
    if (lane == 0) {
      al[k] = alpha;
      tl[k] = tau;
    }
    __syncwarp();
    if (k + 1 < r) {
      double sg2 = 0.0;
      for (int j = k + 2 + lane; j < r; j += 32) {
        const double v = Ms[k + ld * j];
        sg2 += v * v;
      }
      sg2 = warp_sum(sg2);
      const double y0 = Ms[k + ld * (k + 1)];
      double tau2 = 0.0, beta = y0;
      if (sg2 > 0.0) {
        const double ny = sqrt(y0 * y0 + sg2);
        beta = (y0 > 0.0) ? -ny : ny;
        tau2 = (beta - y0) / beta;
        const double iv = 1.0 / (y0 - beta);
        for (int j = k + 2 + lane; j < r; j += 32) Ms[k + ld * j] *= iv;
      }
      __syncwarp();
      if (tau2 != 0.0) {
        for (int i = k + 1 + lane; i < r; i += 32) {
          double sv = Ms[i + ld * (k + 1)];
          for (int j = k + 2; j < r; ++j) sv += Ms[i + ld * j] * Ms[k + ld * j];
          sv *= tau2;
          Ms[i + ld * (k + 1)] -= sv;
          for (int j = k + 2; j < r; ++j) Ms[i + ld * j] -= sv * Ms[k + ld * j];
        }
      }
      if (lane == 0) {
        be[k + 1] = beta;
        tr[k] = tau2;
      }
      __syncwarp();
    }
  }
  __syncwarp();
  for (int q = lane; q < L.total; q += 32) Sg[q] = sm[q];
  (void)Ro;
}

// Sturm count of the scaled Golub-Kahan tridiagonal (squared scaled off-diagonal
// e2[0..m-2]), one thread: two FP64 operations per step (the sign tests read the
// sign and exponent bits on the integer pipe).
__device__ int sturm_count_gk(const double* e2, int m, double x) {
  double d0 = 1.0, d1 = -x;
  bool neg_prev = __double_as_longlong(d1) < 0 && d1 != 0.0;
  int cnt = neg_prev ? 1 : 0;
  for (int k = 2; k <= m; ++k) {
    const double d2 = fma(-x, d1, -e2[k - 2] * d0);
    const long long bits = __double_as_longlong(d2);
    // a zero minor counts as a sign change
    const bool neg = ((bits << 1) == 0) ? !neg_prev : (bits < 0);
    cnt += (neg != neg_prev) ? 1 : 0;
    neg_prev = neg;
    d0 = d1;
    d1 = d2;
    if ((k & 31) == 0) {
      // rescale when both minors are tiny (exponent field below that of 1e-200)
      const int ex1 = (int)((__double_as_longlong(d1) >> 52) & 0x7ff);
      const int ex0 = (int)((__double_as_longlong(d0) >> 52) & 0x7ff);
      if (ex1 < 358 && ex0 < 358) {
        d0 *= 1e200;
        d1 *= 1e200;
      }
    }
  }
  return cnt;
}

// per-thread shared-memory work of k_ksvd_tri (doubles): squared off-diagonal, the
// three U diagonals, the L multipliers, the vector (6 m) and the pivots (m ints); odd so
// that the 32 threads' regions start in different banks
__host__ __device__ inline int tri_stride(int m) { return (6 * m + (m + 1) / 2 + 1) | 1; }

__global__ void __launch_bounds__(32) k_ksvd_tri(KsvdArgs A) {
  extern __shared__ double smt[];
  const int n = A.n, rz = A.rz, r = n + rz;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t e = t >> 1;
  const int k = (int)(t & 1);
  if (e >= A.E) return;
  if (A.mask && !A.mask[e]) return;
  const KsvdSmem L = ksvd_smem(n, rz);
  double* S = A.scr + (size_t)e * ksvd_scr_stride(n, rz);
  const double *al = S + L.al, *be = S + L.be;
  const int J = r, m = 2 * J;
  if (k >= J) {
    S[L.scal + k] = 0.0;
    return;
  }
  // the recurrences below are chains of dependent steps: their operands live in shared
  // memory, not in the global scratch (an L2 round trip per step)
  double* my = smt + (size_t)threadIdx.x * tri_stride(m);
  double* e2 = my;                             // squared scaled off-diagonal
  double* w0 = my + m;                         // d, du, du2
  double* dl = my + 4 * m;                     // off-diagonal, then the L multipliers
  double* zs = my + 5 * m;
  int* piv = reinterpret_cast<int*>(my + 6 * m);
  double bnd = 0.0;
  for (int i = 0; i < m; ++i) {
    const double a = (i > 0) ? fabs(((i - 1) & 1) ? be[i >> 1] : al[(i - 1) >> 1]) : 0.0;
    const double b = (i < m - 1) ? fabs((i & 1) ? be[(i + 1) >> 1] : al[i >> 1]) : 0.0;
    bnd = fmax(bnd, a + b);
  }
  if (bnd == 0.0) bnd = 1.0;
  const double ib = 1.0 / bnd;
  // bisection for the (m - k)-th smallest eigenvalue of the scaled tridiagonal in [0, 1]
  // (to 2^-30 of the bound: the shift of the inverse iteration below; the value
  // itself is the Rayleigh quotient of the converged vector, accurate to the
  // square of the vector's error)
  const int idx = m - k;
  for (int i = 0; i < m - 1; ++i) {
    const double es = ((i & 1) ? be[(i + 1) >> 1] : al[i >> 1]) * ib;
    e2[i] = es * es;
  }
  double lo = 0.0, hi = 1.0 + 1e-12;
  for (int it = 0; it < 30; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count_gk(e2, m, mid) >= idx) hi = mid;
    else lo = mid;
  }
  const double lam = 0.5 * (lo + hi) * bnd;
  // eigenvector by inverse iteration on the unscaled tridiagonal (dl starts as the
  // off-diagonal, which the factorisation reads entry by entry before overwriting it)
  for (int i = 0; i < m - 1; ++i) dl[i] = (i & 1) ? be[(i + 1) >> 1] : al[i >> 1];
  for (int i = 0; i < m; ++i) zs[i] = splitmix_unit(300 + k, i);
  inverse_iteration(dl, m, lam, zs, w0, w0 + m, w0 + 2 * m, dl, piv, kEps * bnd + 1e-300);
  // Rayleigh quotient z^T T z = 2 sum_i ee_i z_i z_{i+1} (|z| = 1; zero diagonal)
  double rq = 0.0;
  for (int i = 0; i < m - 1; ++i) rq = fma((i & 1) ? be[(i + 1) >> 1] : al[i >> 1], zs[i] * zs[i + 1], rq);
  double* z = S + (k ? L.z2 : L.z1);
  for (int i = 0; i < m; ++i) z[i] = zs[i];
  S[L.scal + k] = 2.0 * rq;
}

__global__ void __launch_bounds__(128) k_ksvd_vec(KsvdArgs A) {
  extern __shared__ double smk[];
  const int n = A.n, rz = A.rz, r = n + rz, nn = n * n, Ro = nn - n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= A.E) return;
  if (A.mask && !A.mask[e]) return;
  const KsvdSmem L = ksvd_smem(n, rz);
  double* sm = smk + (size_t)warp * L.total;
  const double* Sg = A.scr + (size_t)e * ksvd_scr_stride(n, rz);
  for (int q = lane; q < L.total; q += 32) sm[q] = Sg[q];
  __syncwarp();
  double* Ms = sm + L.M;
  const int ld = L.ldm;
  double *z1 = sm + L.z1, *z2 = sm + L.z2, *tl = sm + L.tl, *tr = sm + L.tr;
  double *mu1 = sm + L.mu1, *mv1 = sm + L.mv1, *mu2 = sm + L.mu2, *mv2 = sm + L.mv2;
  double* scal = sm + L.scal;
  const int64_t base = e * nn;
  const int J = r, m = 2 * J;
  if (J >= 2) {         // z2 orthogonal to z1 (matters if sigma_1 ~ sigma_2)
    double dt = 0.0;
    for (int i = lane; i < m; i += 32) dt += z1[i] * z2[i];
    dt = warp_sum(dt);
    double nr = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double v = z2[i] - dt * z1[i];
      z2[i] = v;
      nr += v * v;
    }
    nr = warp_sum(nr);
    const double inr = 1.0 / sqrt(nr);
    for (int i = lane; i < m; i += 32) z2[i] *= inr;
    __syncwarp();
  }
  const int nsv = (J >= 2) ? 2 : 1;
  // ---- singular vectors in M coordinates: u = U_h u', v = V_h v' (u' from the
  // odd, v' from the even entries of z), reflectors applied last to first;
  // gauge trace(A_k) >= 0.  The four back-transformations are independent: one
  // per group of 8 lanes (g = 0: u_1, 1: u_2 by the left reflectors; 2: v_1,
  // 3: v_2 by the right ones).
  {
    const int g = lane >> 3, gl = lane & 7, k = g & 1;
    const bool left = g < 2;
    const double* z = k ? z2 : z1;
    double* vec = left ? (k ? mu2 : mu1) : (k ? mv2 : mv1);
    const bool act = k < nsv;
    for (int t = gl; t < r; t += 8) vec[t] = act ? z[2 * t + (left ? 1 : 0)] : 0.0;
    __syncwarp();
    for (int q = r - 1; q >= 0; --q) {
      const double tau = left ? tl[q] : ((q + 1 < r) ? tr[q] : 0.0);
      const bool on = act && tau != 0.0;
      const int st0 = left ? q + 1 : q + 2, h = left ? q : q + 1;
      double dt = 0.0;
      if (on)
        for (int i = st0 + gl; i < r; i += 8)
          dt += (left ? Ms[i + ld * q] : Ms[q + ld * i]) * vec[i];
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
      if (on) {
        const double f = tau * (dt + vec[h]);
        for (int i = st0 + gl; i < r; i += 8)
          vec[i] -= f * (left ? Ms[i + ld * q] : Ms[q + ld * i]);
        __syncwarp(0xffu << (8 * g));
        if (gl == 0) vec[h] -= f;
      }
      __syncwarp();
    }
    double p2 = 0.0, trc = 0.0;
    for (int t = gl; t < r; t += 8) {
      p2 += vec[t] * vec[t];
      if (A.qtr) trc += vec[t] * __ldg(A.qtr + t);
      else if (t < n) trc += vec[t];
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      p2 += __shfl_xor_sync(0xffffffffu, p2, o);
      trc += __shfl_xor_sync(0xffffffffu, trc, o);
    }
    // the sign of u_k's trace also flips v_k: group g + 2 takes it from group g
    const double trk = __shfl_sync(0xffffffffu, trc, (left ? g : g - 2) * 8);
    const double sgn = (trk < 0.0) ? -1.0 : 1.0;
    const double fsc = act ? sgn * rsqrt(p2) : 0.0;
    for (int t = gl; t < r; t += 8) vec[t] *= fsc;
    __syncwarp();
  }
  const double s1 = scal[0], s2 = (nsv == 2) ? scal[1] : 0.0;
  // ---- factors A_k, B_k (n x n column-major): u = Q m_u, A_k = sqrt(s_k) mat(u)
  {
    const double r1 = sqrt(s1), r2 = sqrt(s2);
    for (int q = lane; q < 4 * nn; q += 32) {
      const int which = q / nn, idx = q % nn;
      const int a = idx % n, b = idx / n;
      const double* mvec = (which == 0) ? mu1 : (which == 1) ? mv1 : (which == 2) ? mu2 : mv2;
      double val;
      if (A.Qb) {
        double sv = 0.0;
        for (int t = 0; t < r; ++t) sv += __ldg(A.Qb + (size_t)t * nn + idx) * mvec[t];
        val = sv;
      } else if (a == b) {
        val = mvec[a];
      } else {
        const int o = b * (n - 1) + (a > b ? a - 1 : a);
        double sv = 0.0;
        for (int t = 0; t < rz; ++t) sv += __ldg(A.Qo + (size_t)t * Ro + o) * mvec[n + t];
        val = sv;
      }
      const double f = (which < 2) ? r1 : r2;
      double* dst = (which == 0) ? A.A1 : (which == 1) ? A.B1 : (which == 2) ? A.A2 : A.B2;
      dst[base + idx] = f * val;
    }
  }
  if (lane == 0) {
    A.sigma[2 * e] = s1;
    A.sigma[2 * e + 1] = s2;
    atomic_min_double(&A.st->min_sigma_ratio, (s1 > 0.0) ? s2 / s1 : 0.0);
  }
}

// ---- k_invert_w --------------------------------------------------------------
struct InvArgs {
  int n;
  int64_t E;
  const double *sigma, *A1, *B1, *A2, *B2;
  double *LAi, *LBi, *C1, *C2, *cond;   // LAi/LBi/C1/C2 staged in the SA/SB/T1/T2 regions
  int32_t* flags;
  DevStatus* st;
};

// The paper inverts A_2 and B_1 (Sec. 4.2).  A rank-2 Kronecker sum is unchanged by
// A_2 -> A_2 + alpha A_1, B_1 -> B_1 - alpha B_2, and A_2 alone can be numerically
// singular while P is well conditioned, so alpha is taken from a short list
// (alpha = t ||A_2|| / ||A_1||, t = 0 first) to minimise cond_1(L_A) cond_1(L_B),
// stopping at the first pair below 1e3.  Rank-1 blocks invert A_1 and B_1.
__global__ void __launch_bounds__(64) k_invert_w(InvArgs A) {
  extern __shared__ double smi[];
  const int n = A.n, nn = n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= A.E) return;
  double* aug0 = smi + (size_t)warp * (4 * nn + 2 * n + 8);
  double* aug1 = aug0 + 2 * nn;
  double* fac = aug1 + 2 * nn;
  const int64_t base = e * nn;
  const double* A1 = A.A1 + base;
  const double* A2 = A.A2 + base;
  const double* B1 = A.B1 + base;
  const double* B2 = A.B2 + base;
  const double s1 = A.sigma[2 * e], s2 = A.sigma[2 * e + 1];
  const bool rank1 = !(s2 > 1e-14 * s1);
  double nA1 = 0.0, nA2 = 0.0;
  for (int q = lane; q < nn; q += 32) {
    nA1 += A1[q] * A1[q];
    nA2 += A2[q] * A2[q];
  }
  nA1 = warp_sum(nA1);
  nA2 = warp_sum(nA2);
  const double ascale = (nA1 > 0.0) ? sqrt(nA2 / nA1) : 0.0;
  const double tlist[7] = {0.0, 0.25, -0.25, 1.0, -1.0, 4.0, -4.0};
  double best = INFINITY, alpha = 0.0;
  int best_i = 0, last_i = -1;
  const int ncand = rank1 ? 1 : 7;
  for (int ci = 0; ci <= ncand; ++ci) {
    int use;
    if (ci < ncand) {
      use = ci;
    } else {
      if (best_i == last_i) break;
      use = best_i;
    }
    const double al = rank1 ? 0.0 : tlist[use] * ascale;
    for (int q = lane; q < 2 * nn; q += 32) {
      const int c = q / n, rr = q % n;
      double va, vb;
      if (c < n) {
        const int idx = rr + n * c;
        va = rank1 ? A1[idx] : A2[idx] + al * A1[idx];
        vb = rank1 ? B1[idx] : B1[idx] - al * B2[idx];
      } else {
        va = vb = (rr == c - n) ? 1.0 : 0.0;
      }
      aug0[q] = va;
      aug1[q] = vb;
    }
    __syncwarp();
    const double na = norm1_warp(aug0, n), nb = norm1_warp(aug1, n);
    const bool sa = warp_gauss_jordan(aug0, n, fac);
    const bool sb = warp_gauss_jordan(aug1, n, fac);
    double cp = na * norm1_warp(aug0 + nn, n) * nb * norm1_warp(aug1 + nn, n);
    if (sa || sb || !(cp < 1e300)) cp = INFINITY;
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
    __syncwarp();
  }
  const double cond = best;
  const int sing = !(cond <= 1e14);
  const bool shifted = (alpha != 0.0);
  const double* LAi = aug0 + nn;
  const double* LBi = aug1 + nn;
  for (int q = lane; q < nn; q += 32) {
    const int rr = q % n, c = q / n;
    double sa = 0.0, sb = 0.0;
    if (!rank1)
      for (int k = 0; k < n; ++k) {
        sa += LAi[rr + n * k] * A1[k + n * c];
        sb += LBi[rr + n * k] * B2[k + n * c];
      }
    A.C1[base + q] = sa;
    A.C2[base + q] = sb;
    A.LAi[base + q] = LAi[q];
    A.LBi[base + q] = LBi[q];
  }
  if (lane == 0) {
    int fl = 0;
    if (shifted) fl |= 1;
    if (rank1) fl |= 2;
    if (sing) fl |= 8;
    A.flags[e] = fl;
    A.cond[e] = cond;
    if (shifted) atomicAdd(&A.st->build_shifted, 1);
    if (rank1) atomicAdd(&A.st->build_rank1, 1);
    if (sing) atomicAdd(&A.st->build_singular, 1);
    if (cond < 1e300) atomic_max_double(&A.st->max_cond, cond);
  }
}

// ---- k_invert_r (n <= 16): the same gauge search with both inversions of a
// candidate in one warp: lanes 0-15 hold the rows of A_2 + alpha A_1, lanes 16-31
// those of B_1 - alpha B_2, and one in-place Gauss-Jordan pass inverts both.  The
// candidates are ranked in FP32 (their condition numbers only choose alpha); the
// chosen pair is then inverted in FP64.

// dual in-place Gauss-Jordan (see warp_gj_inplace) of two m x m matrices, m <= 16,
// one per half-warp; pivot rows of step k in bits 4k..4k+3 of piv; returns kr.
template <typename T>
__device__ __forceinline__ int warp_gj_dual(T (&a)[16], uint64_t& piv, int m, bool& sing) {
  const int lane = threadIdx.x & 31, row = lane & 15, hb = lane & 16;
  bool used = row >= m;
  int kr = -1;
  piv = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < m) {
      const int key = used ? -1 : mag_key(a[k]);
      int mx = key;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const unsigned b1 = __ballot_sync(0xffffffffu, !used && key == mx);
      const unsigned b2 = __ballot_sync(0xffffffffu, !used);
      if (mx <= 0) sing = true;
      const unsigned bits = ((mx > 0 ? b1 : b2) >> hb) & 0xffffu;
      const int p = __ffs(bits) - 1;
      const int src = hb + p;
      const T pv = __shfl_sync(0xffffffffu, a[k], src);
      const T ip = (pv != T(0)) ? T(1) / pv : T(0);
      const bool isp = (row == p);
      const T f = a[k] * ip;
      const T s1 = isp ? ip : -f;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (c == k || c >= m) continue;
        const T v = __shfl_sync(0xffffffffu, a[c], src);
        a[c] = fma(s1, v, isp ? T(0) : a[c]);
      }
      a[k] = s1;
      if (isp) {
        used = true;
        kr = k;
      }
      piv |= (uint64_t)p << (4 * k);
    }
  }
  return kr;
}

// 1-norms (max column sums of |.|) of the half-warp's matrix and of its inverse slots
template <typename T>
__device__ __forceinline__ float half_norm1(const T (&a)[16], int m) {
  float best = 0.0f;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if (c >= m) continue;
    float v = fabsf((float)a[c]);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    best = fmaxf(best, v);
  }
  return best;
}

template <typename T>
__device__ __forceinline__ void invert_rows_load(const InvArgs& A, int64_t base, bool rank1,
                                                 double al, T (&a)[16]) {
  const int lane = threadIdx.x & 31, row = lane & 15, n = A.n;
  const bool bside = lane >= 16;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    double v = 0.0;
    if (row < n && c < n) {
      const int64_t idx = base + row + n * c;
      if (!bside) v = rank1 ? A.A1[idx] : A.A2[idx] + al * A.A1[idx];
      else v = rank1 ? A.B1[idx] : A.B1[idx] - al * A.B2[idx];
    }
    a[c] = (T)v;
  }
}

// cond_1 product of a candidate from the two halves' norms (double: no overflow)
__device__ __forceinline__ double pair_cond(float nm, float ninv, bool sing) {
  const int lane = threadIdx.x & 31;
  const double mine = (double)nm * (double)ninv;
  const double other = __shfl_xor_sync(0xffffffffu, mine, 16);
  const bool anys = __any_sync(0xffffffffu, sing);
  const double cp = mine * other;
  (void)lane;
  return (anys || !(cp < 1e300)) ? INFINITY : cp;
}

__global__ void __launch_bounds__(128, 4) k_invert_r(InvArgs A) {
  const int n = A.n, nn = n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, row = lane & 15;
  const bool bside = lane >= 16;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= A.E) return;
  const int64_t base = e * nn;
  const double s1 = A.sigma[2 * e], s2 = A.sigma[2 * e + 1];
  const bool rank1 = !(s2 > 1e-14 * s1);
  double nA1 = 0.0, nA2 = 0.0;
  for (int q = lane; q < nn; q += 32) {
    nA1 += A.A1[base + q] * A.A1[base + q];
    nA2 += A.A2[base + q] * A.A2[base + q];
  }
  nA1 = warp_sum(nA1);
  nA2 = warp_sum(nA2);
  const double ascale = (nA1 > 0.0) ? sqrt(nA2 / nA1) : 0.0;
  double best = INFINITY, alpha = 0.0;
  const int ncand = rank1 ? 1 : 7;
  for (int ci = 0; ci < ncand; ++ci) {
    // t = 0, 0.25, -0.25, 1, -1, 4, -4 (the list of k_invert_w)
    const double t = (ci == 0) ? 0.0 : ((ci & 1) ? 1.0 : -1.0) * ldexp(0.25, 2 * ((ci - 1) >> 1));
    const double al = rank1 ? 0.0 : t * ascale;
    float af[16];
    invert_rows_load<float>(A, base, rank1, al, af);
    const float nm = half_norm1(af, n);
    uint64_t pv;
    bool sg = false;
    warp_gj_dual<float>(af, pv, n, sg);
    const double cp = pair_cond(nm, half_norm1(af, n), sg);
    if (cp < best) {
      best = cp;
      alpha = al;
    }
    if (best <= 1e3) break;
  }
  // the chosen pair in FP64
  double ad[16];
  invert_rows_load<double>(A, base, rank1, alpha, ad);
  const float nm = half_norm1(ad, n);
  uint64_t piv;
  bool sg = false;
  const int kr = warp_gj_dual<double>(ad, piv, n, sg);
  const double cond = pair_cond(nm, half_norm1(ad, n), sg);
  const int sing = !(cond <= 1e14);
  const bool shifted = (alpha != 0.0);
  // lane (row r, side): row kr of L_A^-1 (side 0) or L_B^-1 (side 1) in slots piv[c]
  double* Li = bside ? A.LBi : A.LAi;
  double* Cout = bside ? A.C2 : A.C1;
  const double* R = bside ? A.B2 : A.A1;       // C_1 = L_A^-1 A_1, C_2 = L_B^-1 B_2
  if (kr >= 0) {
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c < n) Li[base + kr + n * (int)((piv >> (4 * c)) & 15u)] = ad[c];
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      if (!rank1) {
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < n) v = fma(ad[c], __ldg(R + base + (int)((piv >> (4 * c)) & 15u) + n * j), v);
      }
      Cout[base + kr + n * j] = v;
    }
  }
  (void)row;
  if (lane == 0) {
    int fl = 0;
    if (shifted) fl |= 1;
    if (rank1) fl |= 2;
    if (sing) fl |= 8;
    A.flags[e] = fl;
    A.cond[e] = cond;
    if (shifted) atomicAdd(&A.st->build_shifted, 1);
    if (rank1) atomicAdd(&A.st->build_rank1, 1);
    if (sing) atomicAdd(&A.st->build_singular, 1);
    if (cond < 1e300) atomic_max_double(&A.st->max_cond, cond);
  }
}

// ---- k_schur_w: real Schur form of C (staged in T1 / T2), one warp per matrix
// (mpe = 2: C_1 and C_2 of every element; mpe = 1: C_1 only)
__global__ void __launch_bounds__(128) k_schur_w(int n, int64_t E, int mpe, double* T1,
                                                 double* T2, double* Q1, double* Q2,
                                                 uint32_t* masks, int32_t* flags, DevStatus* st) {
  extern __shared__ double sms[];
  const int nn = n * n, ld = ld_of(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mtx = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (mtx >= mpe * E) return;
  const int64_t e = mtx / mpe;
  const int which = (int)(mtx % mpe);
  double* H = sms + (size_t)warp * (2 * n * ld + 32);
  double* Q = H + n * ld;
  double* vb = Q + n * ld;
  double* Tg = (which ? T2 : T1) + e * nn;
  double* Qg = (which ? Q2 : Q1) + e * nn;
  const bool rank1 = (flags[e] & 2) != 0;
  for (int q = lane; q < nn; q += 32) {
    const int rr = q % n, c = q / n;
    H[rr + ld * c] = rank1 ? ((which && rr == c) ? 1.0 : 0.0) : Tg[q];
  }
  __syncwarp();
  bool ok = true, relaxed = false;
  if (rank1) {     // P = A1 (x) B1: T1 = 0, T2 = I, Q = I
    for (int q = lane; q < nn; q += 32) {
      const int rr = q % n, c = q / n;
      Q[rr + ld * c] = (rr == c) ? 1.0 : 0.0;
    }
    __syncwarp();
  } else {
    ok = warp_real_schur(H, Q, n, ld, vb, &relaxed);
  }
  for (int q = lane; q < nn; q += 32) {
    const int rr = q % n, c = q / n;
    Tg[q] = H[rr + ld * c];
    Qg[q] = Q[rr + ld * c];
  }
  if (lane == 0) {
    uint32_t m = 0;
    for (int i = 0; i + 1 < n; ++i)
      if (H[(i + 1) + ld * i] != 0.0) m |= 1u << i;
    masks[2 * e + which] = m;
    if (mpe == 1) masks[2 * e + 1] = 0u;
    if (!ok) {
      atomicOr(reinterpret_cast<int*>(flags + e), 4);
      atomicAdd(&st->build_schur_fail, 1);
    } else if (relaxed) {
      atomicOr(reinterpret_cast<int*>(flags + e), 16);
      atomicAdd(&st->build_schur_relaxed, 1);
    }
  }
}

// ---- k_schur_w2: k_schur_w with two matrices per warp (n <= 16)
__global__ void __launch_bounds__(128) k_schur_w2(int n, int64_t E, int mpe, double* T1,
                                                  double* T2, double* Q1, double* Q2,
                                                  uint32_t* masks, int32_t* flags, DevStatus* st) {
  extern __shared__ double sms[];
  const int nn = n * n, ld = ld_of(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, hl = lane & 15, h = lane >> 4;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (2 * gw >= mpe * E) return;                     // whole warp
  const int64_t mtx = 2 * gw + h;
  const bool empty = mtx >= mpe * E;
  const int64_t e = empty ? 0 : mtx / mpe;
  const int which = empty ? 0 : (int)(mtx % mpe);
  double* H = sms + (size_t)(2 * warp + h) * (2 * n * ld + 16);
  double* Q = H + n * ld;
  double* vb = sms + (size_t)8 * (2 * n * ld + 16) + (size_t)warp * 32;
  double* Tg = (which ? T2 : T1) + e * nn;
  double* Qg = (which ? Q2 : Q1) + e * nn;
  const bool rank1 = empty || (flags[e] & 2) != 0;
  for (int c = 0; c < n; ++c)
    if (hl < n) H[hl + ld * c] = rank1 ? ((which && hl == c && !empty) ? 1.0 : 0.0) : Tg[hl + n * c];
  __syncwarp();
  bool relaxed = false;
  const bool ok = hw_real_schur(H, Q, n, ld, vb, rank1, &relaxed);
  // 2x2 diagonal blocks with real eigenvalues are rotated to upper triangular form
  // (Givens rotation whose first column is an eigenvector), so that only complex
  // pairs stay 2x2; kept when the rotated block does not come out triangular to
  // rounding (nearly equal eigenvalues)
  for (int j = 0; j + 1 < n; ++j) {
    const double t00 = H[j + ld * j], t01 = H[j + ld * (j + 1)];
    const double t10 = H[(j + 1) + ld * j], t11 = H[(j + 1) + ld * (j + 1)];
    const bool start = t10 != 0.0 && (j == 0 || H[j + ld * (j - 1)] == 0.0);
    const double hd = 0.5 * (t00 - t11), disc = hd * hd + t01 * t10;
    bool rot = start && ok && !rank1 && disc > 0.0;
    double cr = 1.0, sr = 0.0;
    if (rot) {
      const double lam = 0.5 * (t00 + t11) + copysign(sqrt(disc), hd);
      // eigenvector of lam: (t01, lam - t00) or (lam - t11, t10), the longer one
      double v0 = t01, v1 = lam - t00;
      const double w0 = lam - t11, w1 = t10;
      if (w0 * w0 + w1 * w1 > v0 * v0 + v1 * v1) {
        v0 = w0;
        v1 = w1;
      }
      const double iv = rsqrt(v0 * v0 + v1 * v1);
      cr = v0 * iv;
      sr = v1 * iv;
      // rotated block G^T B G, G = [[c, -s], [s, c]] (first column the eigenvector):
      // its (1, 0) entry g2^T B g1 must vanish to rounding
      const double r10 = -sr * (cr * t00 + sr * t01) + cr * (cr * t10 + sr * t11);
      const double r00 = cr * (cr * t00 + sr * t01) + sr * (cr * t10 + sr * t11);
      const double r11 = -sr * (-sr * t00 + cr * t01) + cr * (-sr * t10 + cr * t11);
      rot = fabs(r10) <= 1e-14 * (fabs(r00) + fabs(r11) + fabs(t01) + fabs(t10));
    }
    __syncwarp();
    if (rot) {
      if (j + hl < n) {                       // rows j, j+1 of columns j..n-1
        const int c = j + hl;
        const double a = H[j + ld * c], bb = H[(j + 1) + ld * c];
        H[j + ld * c] = cr * a + sr * bb;
        H[(j + 1) + ld * c] = -sr * a + cr * bb;
      }
    }
    __syncwarp();
    if (rot) {
      if (hl < n) {                           // columns j, j+1 of rows 0..j+1, and of Q
        const int r = hl;
        if (r <= j + 1) {
          const double a = H[r + ld * j], bb = H[r + ld * (j + 1)];
          H[r + ld * j] = cr * a + sr * bb;
          H[r + ld * (j + 1)] = -sr * a + cr * bb;
        }
        const double qa = Q[r + ld * j], qb = Q[r + ld * (j + 1)];
        Q[r + ld * j] = cr * qa + sr * qb;
        Q[r + ld * (j + 1)] = -sr * qa + cr * qb;
      }
    }
    __syncwarp();
    if (rot && hl == 0) H[(j + 1) + ld * j] = 0.0;
    __syncwarp();
  }
  if (!empty) {
    for (int c = 0; c < n; ++c)
      if (hl < n) {
        Tg[hl + n * c] = H[hl + ld * c];
        Qg[hl + n * c] = Q[hl + ld * c];
      }
    if (hl == 0) {
      uint32_t m = 0;
      for (int i = 0; i + 1 < n; ++i)
        if (H[(i + 1) + ld * i] != 0.0) m |= 1u << i;
      masks[2 * e + which] = m;
      if (mpe == 1) masks[2 * e + 1] = 0u;
      if (!ok && !rank1) {
        atomicOr(reinterpret_cast<int*>(flags + e), 4);
        atomicAdd(&st->build_schur_fail, 1);
      } else if (relaxed && !rank1) {
        atomicOr(reinterpret_cast<int*>(flags + e), 16);
        atomicAdd(&st->build_schur_relaxed, 1);
      }
    }
  }
}

// ---- k_final_w: S_A = Q1^T L_A^-1, S_B = Q2^T L_B^-1 (in place over the staged inverses)
// (mpe = 2: both; mpe = 1: S_A only)
__global__ void __launch_bounds__(128) k_final_w(int n, int64_t E, int mpe, double* SA,
                                                 double* SB, const double* Q1, const double* Q2) {
  extern __shared__ double smf[];
  const int nn = n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mtx = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (mtx >= mpe * E) return;
  const int64_t e = mtx / mpe;
  const int which = (int)(mtx % mpe);
  double* Qs = smf + (size_t)warp * 2 * nn;
  double* Ls = Qs + nn;
  double* S = (which ? SB : SA) + e * nn;
  const double* Qg = (which ? Q2 : Q1) + e * nn;
  for (int q = lane; q < nn; q += 32) {
    Qs[q] = Qg[q];
    Ls[q] = S[q];
  }
  __syncwarp();
  for (int q = lane; q < nn; q += 32) {
    const int rr = q % n, c = q / n;
    double sv = 0.0;
    for (int k = 0; k < n; ++k) sv += Qs[k + n * rr] * Ls[k + n * c];
    S[q] = sv;
  }
}

// ---- k_shift_inv_w: one-sided form of the quasi-triangular system.  With
// C_1 = Q_1 T_1 Q_1^T only (C_2 left unreduced), (C_1 (x) I + I (x) C_2) vec(X)
// = vec(R) becomes C_2 Z + Z T_1^T = R Q_1, Z = X Q_1, solved column block by
// column block from the last: for a 1x1 diagonal block j of T_1,
// (C_2 + T_1[j, j] I) z_j = r_j - sum_{l > j} T_1[j, l] z_l; for a 2x2 block
// {j, j+1} the 2n x 2n system [[C_2 + t00 I, t01 I], [t10 I, C_2 + t11 I]].
// This kernel inverts those diagonal systems (Gauss-Jordan with partial
// pivoting, one warp per element) and stores, for every column j, the n x n
// blocks Gs_j (own column) and Gp_j (partner column of its 2x2 block, zero for
// 1x1): G[e][j][s][k][i], i fastest.  Rank-1 elements (C_1 = 0, C_2 = I)
// store G = I.
// entry (r, c) of the shifted system of the column block at j (size m = n or 2n)
__device__ __forceinline__ double shifted_entry(const double* Tg, const double* Cg, bool rank1,
                                                int n, int j, int r, int c) {
  const int br = r / n, rr = r % n, bc = c / n, cc = c % n;
  const double t = Tg[(j + br) + n * (j + bc)];
  const double c2 = rank1 ? ((rr == cc) ? 1.0 : 0.0) : Cg[rr + n * cc];
  return ((br == bc) ? c2 : 0.0) + ((rr == cc) ? t : 0.0);
}

// G entry for row `row`, column `col` of the inverse of the block at j
__device__ __forceinline__ size_t g_index(int n, int j, int row, int col) {
  const int nn = n * n, a = row / n, i = row % n, bc = col / n, k = col % n;
  return ((size_t)(j + a) * 2 + (bc != a ? 1 : 0)) * nn + (size_t)k * n + i;
}

// Invert the shifted system of the column block at j (size m) and store its
// rows in G.  Kept out of line: inside the block loop of the caller the fully
// unrolled elimination would otherwise not stay in registers.
template <int M, typename T = double>
__device__ __noinline__ bool shift_inv_block(const double* Tg, const double* Cg, bool rank1, int n,
                                             int j, int m, T* Ge) {
  const int lane = threadIdx.x & 31;
  bool sing = false;
  T a[M];
  int piv[M];
#pragma unroll
  for (int c = 0; c < M; ++c)
    a[c] = (lane < m && c < m) ? (T)shifted_entry(Tg, Cg, rank1, n, j, lane, c) : T(0);
  const int kr = warp_gj_inplace<M, T>(a, piv, m, sing);
  if (kr >= 0) {
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < m) Ge[g_index(n, j, kr, piv[c])] = a[c];
  }
  return sing;
}

// 2x2 block {j, j+1} of T_1 with complex eigenvalues (n <= 16).  Balanced by
// D = diag(1, d) (|t01 d| = |t10 / d|), T' = D^-1 T D = W diag(mu, conj mu) W^-1 with
// w = (t01', mu - t00) the eigenvector of mu, the 2n x 2n system
// K = I (x) C_2 + T (x) I has K^-1 = (DW (x) I) diag(Y, conj Y) ((DW)^-1 (x) I),
// Y = (C_2 + mu I)^-1, so block (a, b) of K^-1 is 2 Re(c_ab Y) with
// c_ab = D_a w_a [W^-1]_{0b} / D_b: one complex n x n inverse instead of a real
// 2n x 2n one.  Returns 0 without writing when the block is not a well-separated
// complex pair (|Im mu| < 0.0316 |t01'|: W near singular); bit 0 = done, bit 1 = singular.
template <typename T = double>
__device__ __noinline__ int shift_inv_pair_c(const double* Tg, const double* Cg, int n, int j,
                                             T* Ge) {
  double t00 = Tg[j + n * j], t01 = Tg[j + n * (j + 1)];
  double t10 = Tg[(j + 1) + n * j], t11 = Tg[(j + 1) + n * (j + 1)];
  if (!(t01 * t10 < 0.0)) return 0;
  double d = sqrt(-t10 / t01);                 // D = diag(1, d)
  double b01 = t01 * d;                        // balanced t01' (|t01'| = |t10'|)
  double hd = 0.5 * (t00 - t11);
  double y2 = -(hd * hd + t01 * t10);
  if (!(y2 > 1e-3 * b01 * b01)) return 0;
  const double x = 0.5 * (t00 + t11), y = sqrt(y2);

  const int lane = threadIdx.x & 31, row = lane & 15;
  const bool im = lane >= 16;
  T a[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    double v = 0.0;
    if (row < n && c < n) v = im ? ((c == row) ? y : 0.0) : Cg[row + n * c] + ((c == row) ? x : 0.0);
    a[c] = (T)v;
  }
  bool sing = false;
  uint64_t piv;
  const int kr = warp_gj_inplace_c<T>(a, piv, n, sing);
  // coefficients (recomputed here to keep them out of the elimination's registers):
  // w = (b01, -hd + i y); 1 / det W = i idet, idet = 1 / (2 y b01);
  // u = [W^-1]_{0.} = ((y - i hd) idet, -i b01 idet); c_ab = D_a w_a u_b / D_b
  t00 = Tg[j + n * j];
  t01 = Tg[j + n * (j + 1)];
  t10 = Tg[(j + 1) + n * j];
  t11 = Tg[(j + 1) + n * (j + 1)];
  d = sqrt(-t10 / t01);
  b01 = t01 * d;
  hd = 0.5 * (t00 - t11);
  const double idet = 1.0 / (2.0 * y * b01);
  const double u0r = y * idet, u0i = -hd * idet, u1i = -b01 * idet;
  // re lanes: blocks (0, 0), (0, 1); im lanes: (1, 0), (1, 1)
  double car0, cai0, car1, cai1;
  if (!im) {
    car0 = b01 * u0r;
    cai0 = b01 * u0i;
    car1 = 0.0;
    cai1 = b01 * u1i / d;
  } else {
    car0 = (-hd * u0r - y * u0i) * d;
    cai0 = (-hd * u0i + y * u0r) * d;
    car1 = -y * u1i;
    cai1 = -hd * u1i;
  }
  const int ab = im ? 1 : 0;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const T own = a[c];
    const T oth = __shfl_xor_sync(0xffffffffu, own, 16);
    if (c < n && kr >= 0) {
      const T yr = im ? oth : own, yi = im ? own : oth;
      const int kc = (int)((piv >> (4 * c)) & 15u);
      Ge[g_index(n, j, ab * n + kr, kc)] = T(2) * ((T)car0 * yr - (T)cai0 * yi);
      Ge[g_index(n, j, ab * n + kr, n + kc)] = T(2) * ((T)car1 * yr - (T)cai1 * yi);
    }
  }
  return 1 | (sing ? 2 : 0);
}

// n <= M / 2: one warp per element.  1x1 blocks: register Gauss-Jordan (lanes
// own rows); 2x2 blocks: the complex form above, else (nearly defective
// blocks) a bit in fb[e] for k_shift_inv_fb, which inverts the real 2n x 2n
// system.
template <int M, typename T = double>
__global__ void __launch_bounds__(128) k_shift_inv_r(int n, int64_t E, const double* T1,
                                                     const double* C2, const uint32_t* masks,
                                                     int32_t* flags, T* G, uint32_t* fb,
                                                     DevStatus* st) {
  const int nn = n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= E) return;
  const double* Tg = T1 + e * nn;
  const double* Cg = C2 + e * nn;
  const bool rank1 = (flags[e] & 2) != 0;
  const uint32_t m1 = masks[2 * e];
  T* Ge = G + (size_t)e * 2 * n * nn;
  // block starts (the same walk as the apply), then Gp of 1x1 blocks is zero
  uint32_t cst = 0;
  for (int r = 0; r < n;) {
    const bool two = ((m1 >> r) & 1u) && r + 1 < n;
    if (two) cst |= 1u << r;
    r += two ? 2 : 1;
  }
  for (int q = lane; q < 2 * n * nn; q += 32) {
    const int j = q / (2 * nn), sblk = (q / nn) & 1;
    const bool pairj = ((cst >> j) & 1u) || (j > 0 && ((cst >> (j - 1)) & 1u));
    if (sblk == 1 && !pairj) Ge[q] = T(0);
  }
  bool sing = false;
  uint32_t fbits = 0;
  int j = 0;
  while (j < n) {
    const bool pair = ((m1 >> j) & 1u) && j + 1 < n;
    if (pair) {
      const int pc = rank1 ? 0 : shift_inv_pair_c<T>(Tg, Cg, n, j, Ge);
      if (pc) sing |= (pc & 2) != 0;
      else fbits |= 1u << j;
    } else {
      sing |= shift_inv_block<M / 2, T>(Tg, Cg, rank1, n, j, n, Ge);
    }
    j += pair ? 2 : 1;
  }
  if (lane == 0) {
    fb[e] = fbits;
    if (sing) {
      atomicOr(reinterpret_cast<int*>(flags + e), 8);
      atomicAdd(&st->build_singular, 1);
    }
  }
}

// the real 2n x 2n inverses of the 2x2 blocks k_shift_inv_r left (bits of fb[e])
template <int M, typename T = double>
__global__ void __launch_bounds__(128) k_shift_inv_fb(int n, int64_t E, const double* T1,
                                                      const double* C2, int32_t* flags, T* G,
                                                      const uint32_t* fb, DevStatus* st) {
  const int nn = n * n;
  const int warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= E) return;
  uint32_t bits = fb[e];
  if (!bits) return;
  const bool rank1 = (flags[e] & 2) != 0;
  bool sing = false;
  while (bits) {
    const int j = __ffs(bits) - 1;
    bits &= bits - 1;
    sing |= shift_inv_block<M, T>(T1 + e * nn, C2 + e * nn, rank1, n, j, 2 * n,
                               G + (size_t)e * 2 * n * nn);
  }
  if ((threadIdx.x & 31) == 0 && sing) {
    atomicOr(reinterpret_cast<int*>(flags + e), 8);
    atomicAdd(&st->build_singular, 1);
  }
}

// n > 16: shared-memory Gauss-Jordan (2n x 2n blocks exceed the register rows)
__global__ void __launch_bounds__(128) k_shift_inv_w(int n, int64_t E, const double* T1,
                                                     const double* C2, const uint32_t* masks,
                                                     int32_t* flags, double* G, DevStatus* st) {
  extern __shared__ double smg[];
  const int nn = n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= E) return;
  double* aug = smg + (size_t)warp * (8 * nn + 2 * n + 8);
  double* fac = aug + 8 * nn;
  const double* Tg = T1 + e * nn;
  const double* Cg = C2 + e * nn;
  const bool rank1 = (flags[e] & 2) != 0;
  const uint32_t m1 = masks[2 * e];
  double* Ge = G + (size_t)e * 2 * n * nn;
  bool sing = false;
  int j = 0;
  while (j < n) {
    const bool pair = ((m1 >> j) & 1u) && j + 1 < n;
    const int m = pair ? 2 * n : n;
    for (int q = lane; q < 2 * m * m; q += 32) {
      const int r = q % m, c = q / m;
      aug[q] = (c < m) ? shifted_entry(Tg, Cg, rank1, n, j, r, c) : ((r == c - m) ? 1.0 : 0.0);
    }
    __syncwarp();
    sing |= warp_gauss_jordan(aug, m, fac);
    const double* inv = aug + (size_t)m * m;
    const int ncols = pair ? 2 : 1;
    for (int q = lane; q < ncols * 2 * nn; q += 32) {
      const int a = q / (2 * nn), sblk = (q / nn) & 1, rem = q % nn, k = rem / n, i = rem % n;
      double v = 0.0;
      if (sblk == 0) v = inv[(a * n + i) + m * (a * n + k)];
      else if (pair) v = inv[(a * n + i) + m * ((1 - a) * n + k)];
      Ge[((size_t)(j + a) * 2 + sblk) * nn + k * n + i] = v;
    }
    __syncwarp();
    j += ncols;
  }
  if (lane == 0 && sing) {
    atomicOr(reinterpret_cast<int*>(flags + e), 8);
    atomicAdd(&st->build_singular, 1);
  }
}

// ---- learned factors: network inputs, normalised cores, acceptance ------------
__global__ void k_coef_2d(const Tables* T, int n, int64_t E, double h, const double* cx,
                          const double* cy, const double* fa, double* kco, const double* mq);

// Mn = M / ||M||_F (column-major r x r) and ||M||_F (= ||A~||_F) per element
__global__ void __launch_bounds__(128) k_core(const double* kco, const double* Zd, const double* Rz,
                                              int n, int rz, int64_t E, double* Mn, double* norms) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= E) return;
  const int nc = n + 2, nn = n * n, r = n + rz;
  const double* kc = kco + (size_t)e * (2 * nc * n + nn);
  double* M = Mn + (size_t)e * r * r;
  form_core(kc, kc + nc * n, kc + 2 * nc * n, Zd, Rz, n, rz, M, r);
  __syncwarp();
  double s2 = 0.0;
  for (int q = lane; q < r * r; q += 32) s2 += M[q] * M[q];
  const double nr = sqrt(warp_sum(s2));
  const double inv = (nr > 0.0) ? 1.0 / nr : 0.0;
  for (int q = lane; q < r * r; q += 32) M[q] *= inv;
  if (lane == 0) norms[e] = nr;
}

// network input of an element: a_x, a_y at the n x n nodes (recovered from the
// scaled flux Jacobians cx = -dt h w_i w_j a_x), then dt / h
__global__ void k_features(const Tables* T, int n, int64_t E, double h, double dt,
                           const double* cx, const double* cy, float* X) {
  const int nn = n * n, K = 2 * nn + 1;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < E * K;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / K;
    const int q = (int)(g % K);
    float v;
    if (q == 2 * nn) {
      v = (float)(dt / h);
    } else {
      const int qq = q % nn, i = qq % n, j = qq / n;
      const double sc = dt * h * T->w[i] * T->w[j];
      const double c = (q < nn ? cx : cy)[e * nn + qq];
      v = (sc > 0.0) ? (float)(-c / sc) : 0.0f;
    }
    X[g] = v;
  }
}

// accept the prediction of element e when sqrt(L_e) <= threshold: factors
// A_k = sqrt(||A~||) * output (column-major), sigma_k = ||A_k|| ||B_k||;
// otherwise flag it for the exact KSVD.
__global__ void __launch_bounds__(128) k_learned_accept(int n, int64_t E, const float* out,
                                                        const double* norms, const double* lossv,
                                                        double threshold, double* A1, double* B1,
                                                        double* A2, double* B2, double* sigma,
                                                        int32_t* mask, DevStatus* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= E) return;
  const int nn = n * n;
  const double err = sqrt(fmax(lossv[e], 0.0));
  const bool ok = err <= threshold;
  if (lane == 0) {
    mask[e] = ok ? 0 : 1;
    if (!ok) atomicAdd(&st->learned_fallback, 1);
  }
  if (!ok) return;
  const double f = sqrt(norms[e]);
  const float* oe = out + (size_t)e * 4 * nn;
  double nk[4] = {0.0, 0.0, 0.0, 0.0};
  double* dst[4] = {A1, B1, A2, B2};
  for (int k = 0; k < 4; ++k) {
    double s2 = 0.0;
    for (int q = lane; q < nn; q += 32) {
      const double v = f * (double)oe[k * nn + q];
      dst[k][(size_t)e * nn + q] = v;
      s2 += v * v;
    }
    nk[k] = sqrt(warp_sum(s2));
  }
  if (lane == 0) {
    const double s1 = nk[0] * nk[1], s2 = nk[2] * nk[3];
    sigma[2 * e] = s1;
    sigma[2 * e + 1] = s2;
    const double hi = fmax(s1, s2);
    atomic_min_double(&st->min_sigma_ratio, (hi > 0.0) ? fmin(s1, s2) / hi : 0.0);
  }
}

size_t ksvd_scr_doubles(int n, int rz) { return ksvd_scr_stride(n, rz); }

cudaError_t launch_learned_inputs(const tpp_ctx* c, float* X, double* Mn, double* norms,
                                  cudaStream_t s) {
  k_coef_2d<<<152 * 4, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->E, c->prob.h,
                                    c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                    c->p<double>(c->L.fa), c->p<double>(c->L.kco),
                                    c->curved ? c->p<double>(c->L.mq) : nullptr);
  count_launch();
  if (Mn) {
    k_core<<<(unsigned)((c->E + 3) / 4), 128, 0, s>>>(c->p<double>(c->L.kco),
                                                      c->p<double>(c->L.zd),
                                                      c->p<double>(c->L.rz), c->n, c->rz, c->E,
                                                      Mn, norms);
    count_launch();
  }
  if (X) {
    k_features<<<152 * 4, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->E, c->prob.h,
                                        c->prob.dt, c->p<double>(c->L.cx),
                                        c->p<double>(c->L.cy), X);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_learned_accept(const tpp_ctx* c, const float* out, const double* norms,
                                  const double* lossv, double threshold, int32_t* mask,
                                  cudaStream_t s) {
  k_learned_accept<<<(unsigned)((c->E + 3) / 4), 128, 0, s>>>(
      c->n, c->E, out, norms, lossv, threshold, c->p<double>(c->L.fA1), c->p<double>(c->L.fB1),
      c->p<double>(c->L.fA2), c->p<double>(c->L.fB2), c->p<double>(c->L.sigma), mask,
      c->p<DevStatus>(c->L.status));
  count_launch();
  return cudaGetLastError();
}

// ---- k_coef_2d: KSVD coefficients of a 2D element block (flux Jacobians of
// Sec. 3.4.1 in the basis of k_struct_qr): Cx[c][j] = cx[c + n j] (volume,
// c < n), max(a.n, 0) on the +x and -x faces (c = n, n + 1); Cy likewise for
// y; Dg[i + n j] = h^2 w_i w_j (mass).
__global__ void k_coef_2d(const Tables* T, int n, int64_t E, double h, const double* cx,
                          const double* cy, const double* fa, double* kco, const double* mq) {
  const int nc = n + 2, nn = n * n, per = 2 * nc * n + nn;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < E * per;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / per;
    const int q = (int)(g % per);
    const double* fe = fa + e * 4 * n;      // outward normal velocities, faces -x, +x, -y, +y
    double v;
    if (q < 2 * nc * n) {
      const int which = q / (nc * n), rem = q % (nc * n);
      const int c = rem / n, j = rem % n;
      if (which == 0) {          // x-part, j = y index
        if (c < n) v = cx[e * nn + c + n * j];
        else if (c == n) v = fmax(fe[1 * n + j], 0.0);       // outflow through +x
        else v = fmax(fe[0 * n + j], 0.0);                   // outflow through -x
      } else {                   // y-part, j = x index
        if (c < n) v = cy[e * nn + j + n * c];
        else if (c == n) v = fmax(fe[3 * n + j], 0.0);
        else v = fmax(fe[2 * n + j], 0.0);
      }
    } else {
      const int d = q - 2 * nc * n, i = d % n, j = d / n;
      v = mq ? mq[e * nn + d] : h * h * T->w[i] * T->w[j];     // mass (curved: w |J_T|)
    }
    kco[g] = v;
  }
}

// KSVD of the 2D-structured blocks in kco (2D elements, or the second stage
// of the 3D nested form), inverses, Schur forms, S_A and S_B.
cudaError_t launch_ksvd_pipeline(const tpp_ctx* c, cudaStream_t s, const int32_t* mask) {
  const int n = c->n;
  const int64_t E = c->E;
  DevStatus* st = c->p<DevStatus>(c->L.status);
  // 1. KSVD
  KsvdArgs ka;
  ka.n = n;
  ka.rz = c->rz;
  ka.E = E;
  ka.kco = c->p<double>(c->L.kco);
  ka.Zd = c->p<double>(c->L.zd);
  ka.Rz = c->p<double>(c->L.rz);
  ka.Qo = c->p<double>(c->L.qo);
  ka.scr = c->p<double>(c->L.bscr);
  ka.iscr = c->p<int>(c->L.biscr);
  ka.sigma = c->p<double>(c->L.sigma);
  ka.A1 = c->p<double>(c->L.fA1);
  ka.B1 = c->p<double>(c->L.fB1);
  ka.A2 = c->p<double>(c->L.fA2);
  ka.B2 = c->p<double>(c->L.fB2);
  ka.st = st;
  ka.mask = mask;
  ka.Mcore = ka.Qb = ka.qtr = nullptr;
  if (c->mu > c->n) {     // over-integration: explicit cores from k_core_mu
    ka.rz = c->r - n;
    ka.Mcore = c->p<double>(c->L.kco);
    ka.Qb = c->p<double>(c->L.qb);
    ka.qtr = c->p<double>(c->L.qtr);
  }
  {
    const int warps = 4;
    const size_t smem = (size_t)warps * ksvd_smem(n, ka.rz).total * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_ksvd_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    k_ksvd_w<<<(unsigned)((E + warps - 1) / warps), warps * 32, smem, s>>>(ka);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // one thread per (element, k): 32-thread CTAs spread the 2 E sequential problems over
    // every SM (the FP64 pipe of an SM, not its warp count, bounds this kernel)
    const size_t tsm = (size_t)32 * tri_stride(2 * (n + ka.rz)) * sizeof(double);
    err = cudaFuncSetAttribute(k_ksvd_tri, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm);
    if (err != cudaSuccess) return err;
    k_ksvd_tri<<<(unsigned)((2 * E + 31) / 32), 32, tsm, s>>>(ka);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_ksvd_vec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_ksvd_vec<<<(unsigned)((E + warps - 1) / warps), warps * 32, smem, s>>>(ka);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return launch_factor_inverse(c, s);
}

// steps 2-5 of the build on the factors A_k, B_k (and sigma) already in the workspace
cudaError_t launch_factor_inverse(const tpp_ctx* c, cudaStream_t s) {
  const int n = c->n, nn = n * n;
  const int64_t E = c->E;
  DevStatus* st = c->p<DevStatus>(c->L.status);
  // 2. inverses and C products
  InvArgs ia;
  ia.n = n;
  ia.E = E;
  ia.sigma = c->p<double>(c->L.sigma);
  ia.A1 = c->p<double>(c->L.fA1);
  ia.B1 = c->p<double>(c->L.fB1);
  ia.A2 = c->p<double>(c->L.fA2);
  ia.B2 = c->p<double>(c->L.fB2);
  ia.LAi = c->p<double>(c->L.fSA);
  ia.LBi = c->p<double>(c->L.fSB);
  ia.C1 = c->p<double>(c->L.fT1);
  ia.C2 = c->p<double>(c->L.fT2);
  ia.cond = c->p<double>(c->L.fSC);
  ia.flags = c->p<int32_t>(c->L.flags);
  ia.st = st;
  if (n <= 16) {
    k_invert_r<<<(unsigned)((E + 3) / 4), 128, 0, s>>>(ia);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  } else {
    const int warps = 2;
    const size_t smem = (size_t)warps * (4 * nn + 2 * n + 8) * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_invert_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    k_invert_w<<<(unsigned)((E + warps - 1) / warps), warps * 32, smem, s>>>(ia);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  // 3. real Schur forms: C_1 and C_2 (two-sided form), or C_1 only
  const bool two = two_sided(c);
  const int mpe = two ? 2 : 1;
  if (n <= 16) {
    const int ld = ld_of(n);
    const size_t smem = ((size_t)8 * (2 * n * ld + 16) + 4 * 32) * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_schur_w2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t warps_needed = (mpe * E + 1) / 2;
    k_schur_w2<<<(unsigned)((warps_needed + 3) / 4), 128, smem, s>>>(
        n, E, mpe, c->p<double>(c->L.fT1), c->p<double>(c->L.fT2), c->p<double>(c->L.fQ1),
        two ? c->p<double>(c->L.fQ2) : nullptr, c->p<uint32_t>(c->L.masks),
        c->p<int32_t>(c->L.flags), st);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  } else   {
    const int warps = 4, ld = ld_of(n);
    const size_t smem = (size_t)warps * (2 * n * ld + 32) * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_schur_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    k_schur_w<<<(unsigned)((mpe * E + warps - 1) / warps), warps * 32, smem, s>>>(
        n, E, mpe, c->p<double>(c->L.fT1), c->p<double>(c->L.fT2), c->p<double>(c->L.fQ1),
        two ? c->p<double>(c->L.fQ2) : nullptr, c->p<uint32_t>(c->L.masks),
        c->p<int32_t>(c->L.flags), st);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  // 4. one-sided form: inverses of the shifted diagonal systems
  if (!two) {
    const double* T1p = c->p<double>(c->L.fT1);
    const double* C2p = c->p<double>(c->L.fT2);
    const uint32_t* mk = c->p<uint32_t>(c->L.masks);
    int32_t* fl = c->p<int32_t>(c->L.flags);
    double* Gp = c->p<double>(c->L.fG);
    cudaError_t err;
    uint32_t* fb = reinterpret_cast<uint32_t*>(c->p<int>(c->L.biscr));   // free after the KSVD
    const unsigned gw = (unsigned)((E + 3) / 4);
    if (c->features & TPP_FEAT_F32_SHIFTS) {   // FP32 inverses straight into the FP32 copies
      float* G32 = c->p<float>(c->L.f32) + f32_layout(n, c->E, c->dim, false).G;
      if (n <= 8) {
        k_shift_inv_r<16, float><<<gw, 128, 0, s>>>(n, E, T1p, C2p, mk, fl, G32, fb, st);
        count_launch();
        k_shift_inv_fb<16, float><<<gw, 128, 0, s>>>(n, E, T1p, C2p, fl, G32, fb, st);
      } else {
        k_shift_inv_r<32, float><<<gw, 128, 0, s>>>(n, E, T1p, C2p, mk, fl, G32, fb, st);
        count_launch();
        k_shift_inv_fb<32, float><<<gw, 128, 0, s>>>(n, E, T1p, C2p, fl, G32, fb, st);
      }
    } else if (n <= 8) {
      k_shift_inv_r<16><<<gw, 128, 0, s>>>(n, E, T1p, C2p, mk, fl, Gp, fb, st);
      count_launch();
      k_shift_inv_fb<16><<<gw, 128, 0, s>>>(n, E, T1p, C2p, fl, Gp, fb, st);
    } else if (n <= 16) {
      k_shift_inv_r<32><<<gw, 128, 0, s>>>(n, E, T1p, C2p, mk, fl, Gp, fb, st);
      count_launch();
      k_shift_inv_fb<32><<<gw, 128, 0, s>>>(n, E, T1p, C2p, fl, Gp, fb, st);
    } else {
      const size_t smem = (size_t)(8 * nn + 2 * n + 8) * sizeof(double);
      err = cudaFuncSetAttribute(k_shift_inv_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
      if (err != cudaSuccess) return err;
      k_shift_inv_w<<<(unsigned)E, 32, smem, s>>>(n, E, T1p, C2p, mk, fl, Gp, st);
    }
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  // 5. S_A = Q_1^T L_A^-1 (and S_B = Q_2^T L_B^-1 in the two-sided form)
  {
    const int warps = 4;
    const size_t smem = (size_t)warps * 2 * nn * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_final_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    k_final_w<<<(unsigned)((mpe * E + warps - 1) / warps), warps * 32, smem, s>>>(
        n, E, mpe, c->p<double>(c->L.fSA), c->p<double>(c->L.fSB), c->p<double>(c->L.fQ1),
        two ? c->p<double>(c->L.fQ2) : nullptr);
    count_launch();
    return cudaGetLastError();
  }
}


cudaError_t launch_build_2d(const tpp_ctx* c, cudaStream_t s) {
  if (c->mu > c->n) {           // over-integrated blocks: explicit cores (k_overint.cu)
    cudaError_t err = launch_core_mu(c, s);
    if (err != cudaSuccess) return err;
    return launch_ksvd_pipeline(c, s, nullptr);
  }
  k_coef_2d<<<152 * 4, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->E, c->prob.h,
                                    c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                    c->p<double>(c->L.fa), c->p<double>(c->L.kco),
                                    c->curved ? c->p<double>(c->L.mq) : nullptr);
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_ksvd_pipeline(c, s, nullptr);
}

// ---------------------------------------------------------------------------
// 3D nested KSVD, stage 1 (Sec. 4.3, Alg. 3d-form step 1): best rank-1
// A ~ A1 (x) D1 of the n^3 x n^3 block, A1 on z.  With collocated quadrature
// the rearrangement A~ (rows: z pairs (k, k'), n^2 x n^4) is E_r X1 + Y1 E_c^T:
// row (k, k) of X1 is vec of the xy block S_k of z slice k (mass, x- and
// y-terms), column (i, j) of Y1 is vec of the z-operator H_ij of the line
// (i, j).  G = A~ A~^T (n^2 x n^2) is applied without forming A~:
//   G u = E_r (P u~ + Sd (Y1^T u)) + Y1 (Sd^T u~ + Y1^T u),
// u~ = E_r^T u, P = X1 X1^T (Gram of the slices), Sd = X1 E_c (their
// diagonals).  P and Sd come from the per-line coefficients in the basis of
// k_struct_qr (off-diagonal parts through Rz, Qo orthonormal), so stage 1
// costs O(n^4) per element.  The top eigenpair of G (symmetric Lanczos with
// full reorthogonalisation) gives sigma_1^2 and u_1; A1 = sqrt(sigma_1)
// mat(u_1) and D1 = (sum_k u~_k S_k + diag(Y1^T u_1)) / sqrt(sigma_1), whose
// coefficients feed the 2D-structured stage 2 (k_ksvd_w).

struct Stage1Args {
  const Tables* T;
  int n, rz, Jmax;
  int64_t E;
  double h;
  const double *cx, *cy, *cz, *fa, *Zd, *Rz;   // fa: [E][6][n^2] outward normal velocities
  double* scr;
  double* kco;
  double *Az, *Azi, *sigz;
  int32_t* zflags;
  DevStatus* st;
};

namespace {

// out = G u for the stage-1 Gram operator (one warp; all arrays global scratch)
__device__ void s1_apply_G(const Tables* T, int n, const double* Cz3, const double* sd,
                           const double* P, const double* u, double* out, double* ut, double* zu,
                           double* yu, double* wv, double* cw) {
  const int lane = threadIdx.x & 31, nn = n * n, nc = n + 2;
  for (int k = lane; k < n; k += 32) ut[k] = u[k + n * k];
  for (int c = lane; c < nc; c += 32) {
    double sv = 0.0;
    if (c < n) {
      for (int a = 0; a < n; ++a) sv += T->D[c * n + a] * u[a + n * c];
    } else {
      const double* lv = (c == n) ? T->l1 : T->l0;
      for (int b = 0; b < n; ++b) {
        double t = 0.0;
        for (int a = 0; a < n; ++a) t += lv[a] * u[a + n * b];
        sv += lv[b] * t;
      }
    }
    zu[c] = sv;
  }
  __syncwarp();
  for (int q = lane; q < nn; q += 32) {
    double y = 0.0;
    for (int c = 0; c < nc; ++c) y += Cz3[(size_t)c * nn + q] * zu[c];
    yu[q] = y;
    double w = y;
    for (int k = 0; k < n; ++k) w += sd[(size_t)k * nn + q] * ut[k];
    wv[q] = w;
  }
  __syncwarp();
  for (int c = lane; c < nc; c += 32) {
    double sv = 0.0;
    for (int q = 0; q < nn; ++q) sv += wv[q] * Cz3[(size_t)c * nn + q];
    cw[c] = sv;
  }
  __syncwarp();
  for (int q = lane; q < nn; q += 32) {
    const int a = q % n, b = q / n;
    double v = T->D[b * n + a] * cw[b] + T->l1[a] * T->l1[b] * cw[n] + T->l0[a] * T->l0[b] * cw[n + 1];
    if (a == b) {
      const int k = a;
      for (int k2 = 0; k2 < n; ++k2) v += P[k + n * k2] * ut[k2];
      for (int r = 0; r < nn; ++r) v += sd[(size_t)k * nn + r] * yu[r];
    }
    out[q] = v;
  }
  __syncwarp();
}

// eigenvalues of the symmetric tridiagonal (diag al, off-diagonal be[1..m-1])
// below x (Sturm count of the LDL^T pivots)
__device__ int sturm_sym(const double* al, const double* be, int m, double x, double tiny) {
  int cnt = 0;
  double q = al[0] - x;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < m; ++i) {
    if (q == 0.0) q = -tiny;
    q = (al[i] - x) - be[i] * be[i] / q;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

}  // namespace

__global__ void __launch_bounds__(128) k_stage1_3d(Stage1Args A) {
  extern __shared__ double sm1[];
  const int n = A.n, nn = n * n, n3 = nn * n, nc = n + 2, rz = A.rz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= A.E) return;
  const S1Layout L = s1_layout(n, rz, A.Jmax);
  double* S = A.scr + (size_t)e * L.total;
  double *Cx3 = S + L.cx3, *Cy3 = S + L.cy3, *Cz3 = S + L.cz3, *rx = S + L.rx, *ry = S + L.ry;
  double *sd = S + L.sd, *P = S + L.P, *Q = S + L.Q, *ut = S + L.ut, *zu = S + L.zu;
  double *yu = S + L.yu, *wv = S + L.wv, *cw = S + L.cw, *tmp = S + L.tmp;
  double *al = S + L.al, *be = S + L.be, *yv = S + L.y;
  double* aug = sm1 + (size_t)warp * (2 * nn + n + 40);
  // per warp: tridiagonal (al, be), the inverse iteration's LU and vector, pivots
  double* tri = sm1 + (size_t)(blockDim.x >> 5) * (2 * nn + n + 40) + (size_t)warp * 520;
  double *als = tri, *bes = tri + 65;
  double* fac = aug + 2 * nn;
  double* cfs = fac + n + 8;   // 32 reorthogonalisation coefficients
  const double* fe = A.fa + e * 6 * nn;      // faces -x, +x, -y, +y, -z, +z
  const double h3 = A.h * A.h * A.h;
  const Tables* T = A.T;
  // ---- 1. line coefficients in the Z basis (flux Jacobians of Sec. 3.4.1)
  for (int q = lane; q < nc * nn; q += 32) {
    const int c = q / nn, t = q % nn, a = t % n, b = t / n;
    double vx, vy, vz;
    if (c < n) {
      vx = A.cx[e * n3 + c + n * a + nn * b];        // x-line (j = a, k = b)
      vy = A.cy[e * n3 + a + n * c + nn * b];        // y-line (i = a, k = b)
      vz = A.cz[e * n3 + a + n * b + nn * c];        // z-line (i = a, j = b)
    } else if (c == n) {        // outflow through the upper faces
      vx = fmax(fe[1 * nn + t], 0.0);
      vy = fmax(fe[3 * nn + t], 0.0);
      vz = fmax(fe[5 * nn + t], 0.0);
    } else {                    // outflow through the lower faces
      vx = fmax(fe[0 * nn + t], 0.0);
      vy = fmax(fe[2 * nn + t], 0.0);
      vz = fmax(fe[4 * nn + t], 0.0);
    }
    Cx3[q] = vx;
    Cy3[q] = vy;
    Cz3[q] = vz;
  }
  __syncwarp();
  // ---- 2. off-diagonal parts through Rz, slice diagonals, Gram P of the slices
  for (int q = lane; q < rz * nn; q += 32) {
    const int t = q / nn, rest = q % nn;
    double a = 0.0, b = 0.0;
    for (int c = 0; c < nc; ++c) {
      const double rzc = __ldg(A.Rz + t * nc + c);
      a += rzc * Cx3[(size_t)c * nn + rest];
      b += rzc * Cy3[(size_t)c * nn + rest];
    }
    rx[q] = a;
    ry[q] = b;
  }
  for (int q = lane; q < n3; q += 32) {
    const int i = q % n, j = (q / n) % n, k = q / nn;
    double v = h3 * T->w[i] * T->w[j] * T->w[k];
    for (int c = 0; c < nc; ++c)
      v += __ldg(A.Zd + i * nc + c) * Cx3[(size_t)c * nn + j + n * k] +
           __ldg(A.Zd + j * nc + c) * Cy3[(size_t)c * nn + i + n * k];
    sd[(size_t)k * nn + i + n * j] = v;
  }
  __syncwarp();
  for (int q = lane; q < nn; q += 32) {
    const int k = q % n, k2 = q / n;
    double v = 0.0;
    for (int t = 0; t < rz; ++t)
      for (int a = 0; a < n; ++a)
        v += rx[(size_t)t * nn + a + n * k] * rx[(size_t)t * nn + a + n * k2] +
             ry[(size_t)t * nn + a + n * k] * ry[(size_t)t * nn + a + n * k2];
    for (int r = 0; r < nn; ++r) v += sd[(size_t)k * nn + r] * sd[(size_t)k2 * nn + r];
    P[q] = v;
  }
  __syncwarp();
  // ---- 3. symmetric Lanczos on G with full reorthogonalisation
  {
    for (int t = lane; t < nn; t += 32) Q[t] = splitmix_unit(7, t);
    __syncwarp();
    double s2 = 0.0;
    for (int t = lane; t < nn; t += 32) s2 += Q[t] * Q[t];
    const double inv = 1.0 / sqrt(warp_sum(s2));
    for (int t = lane; t < nn; t += 32) Q[t] *= inv;
    if (lane == 0) be[0] = 0.0;
    __syncwarp();
  }
  int J = 0;
  double lam = 0.0;
  bool conv = false;
  const int Jmax = A.Jmax;
  double gscale = 0.0;
  for (int j = 0; j < Jmax; ++j) {
    double* qj = Q + (size_t)j * nn;
    double* w = Q + (size_t)(j + 1) * nn;
    s1_apply_G(T, n, Cz3, sd, P, qj, w, ut, zu, yu, wv, cw);
    double a = 0.0;
    for (int t = lane; t < nn; t += 32) a += qj[t] * w[t];
    a = warp_sum(a);
    for (int t = lane; t < nn; t += 32) w[t] -= a * qj[t] + ((j > 0) ? be[j] * Q[(size_t)(j - 1) * nn + t] : 0.0);
    __syncwarp();
    warp_reorth(w, Q, j + 1, nn, cfs);
    double b2 = 0.0;
    for (int t = lane; t < nn; t += 32) b2 += w[t] * w[t];
    const double b = sqrt(warp_sum(b2));
    gscale = fmax(gscale, fabs(a) + b);
    if (lane == 0) {
      al[j] = a;
      be[j + 1] = b;
    }
    J = j + 1;
    const bool breakdown = !(b > 1e-13 * gscale);
    if (!breakdown) {
      const double ib = 1.0 / b;
      for (int t = lane; t < nn; t += 32) w[t] *= ib;
    }
    __syncwarp();
    const bool check = breakdown || J == Jmax || J == nn || (J >= 8 && (J % 8) == 0);
    if (!check) continue;
    // top eigenvalue of the J x J tridiagonal by 32-point multisection; the tridiagonal
    // and the inverse iteration's work sit in this warp's shared memory (their recurrences
    // are chains of dependent steps)
    for (int i = lane; i <= J; i += 32) {
      if (i < J) als[i] = al[i];
      bes[i] = be[i];
    }
    __syncwarp();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < J; ++i) {
      const double rad = ((i > 0) ? fabs(bes[i]) : 0.0) + ((i + 1 < J) ? fabs(bes[i + 1]) : 0.0);
      lo = fmin(lo, als[i] - rad);
      hi = fmax(hi, als[i] + rad);
    }
    const double tiny = 1e-300 + kEps * fmax(fabs(lo), fabs(hi));
    for (int it = 0; it < 12; ++it) {
      const double x = lo + (hi - lo) * (double)(lane + 1) * (1.0 / 33.0);
      const int cnt = sturm_sym(als, bes, J, x, tiny);
      const unsigned ge = __ballot_sync(0xffffffffu, cnt >= J);
      const int f = ge ? (__ffs(ge) - 1) : 32;
      const double wdt = hi - lo;
      const double nlo = (f == 0) ? lo : lo + wdt * (double)f * (1.0 / 33.0);
      const double nhi = (f == 32) ? hi : lo + wdt * (double)(f + 1) * (1.0 / 33.0);
      lo = nlo;
      hi = nhi;
    }
    lam = 0.5 * (lo + hi);
    // eigenvector by inverse iteration (lane 0; tridiagonal with pivoting)
    if (lane == 0) {
      double *d = tri + 130, *du = tri + 194, *du2 = tri + 258, *dl = tri + 322;
      double* ys = tri + 386;
      int* pv = reinterpret_cast<int*>(tri + 450);
      for (int i = 0; i < J; ++i) {
        d[i] = als[i] - lam;
        du[i] = (i + 1 < J) ? bes[i + 1] : 0.0;
        dl[i] = (i + 1 < J) ? bes[i + 1] : 0.0;
        du2[i] = 0.0;
        pv[i] = 0;
        ys[i] = splitmix_unit(11, i);
      }
      for (int i = 0; i + 1 < J; ++i) {
        if (fabs(d[i]) >= fabs(dl[i])) {
          if (d[i] == 0.0) d[i] = tiny;
          const double f = dl[i] / d[i];
          dl[i] = f;
          d[i + 1] -= f * du[i];
        } else {
          const double f = d[i] / dl[i];
          d[i] = dl[i];
          dl[i] = f;
          const double t = du[i];
          du[i] = d[i + 1];
          d[i + 1] = t - f * d[i + 1];
          if (i + 2 < J) {
            du2[i] = du[i + 1];
            du[i + 1] = -f * du[i + 1];
          }
          pv[i] = 1;
        }
      }
      if (d[J - 1] == 0.0) d[J - 1] = tiny;
      for (int it = 0; it < 3; ++it) {
        for (int i = 0; i + 1 < J; ++i) {
          if (pv[i]) {
            const double t = ys[i];
            ys[i] = ys[i + 1];
            ys[i + 1] = t;
          }
          ys[i + 1] -= dl[i] * ys[i];
        }
        for (int i = J - 1; i >= 0; --i) {
          double sv = ys[i];
          if (i + 1 < J) sv -= du[i] * ys[i + 1];
          if (i + 2 < J) sv -= du2[i] * ys[i + 2];
          ys[i] = sv / d[i];
        }
        double nr = 0.0;
        for (int i = 0; i < J; ++i) nr += ys[i] * ys[i];
        nr = 1.0 / sqrt(nr);
        for (int i = 0; i < J; ++i) ys[i] *= nr;
      }
      for (int i = 0; i < J; ++i) yv[i] = ys[i];
      tmp[0] = (breakdown ? 0.0 : bes[J]) * fabs(ys[J - 1]);   // Ritz residual
    }
    __syncwarp();
    conv = breakdown || tmp[0] <= 1e-14 * fabs(lam) || J == nn;
    if (conv || J == Jmax) break;
  }
  // ---- 4. u_1, A1 and the stage-2 coefficients of D1
  for (int t = lane; t < nn; t += 32) {
    double sv = 0.0;
    for (int i = 0; i < J; ++i) sv += yv[i] * Q[(size_t)i * nn + t];
    tmp[t] = sv;
  }
  __syncwarp();
  double nr = 0.0, tr = 0.0;
  for (int t = lane; t < nn; t += 32) {
    nr += tmp[t] * tmp[t];
    if (t % (n + 1) == 0) tr += tmp[t];
  }
  nr = warp_sum(nr);
  tr = warp_sum(tr);
  const double sgn = (tr < 0.0) ? -1.0 : 1.0;          // gauge: trace(A1) >= 0
  const double fu = sgn / sqrt(nr);
  for (int t = lane; t < nn; t += 32) tmp[t] *= fu;
  __syncwarp();
  const double s1 = sqrt(fmax(lam, 0.0));
  const double rs = sqrt(s1), irs = (rs > 0.0) ? 1.0 / rs : 0.0;
  for (int t = lane; t < nn; t += 32) A.Az[e * nn + t] = rs * tmp[t];
  // Y1^T u_1 (into yu) and u~ (ut) with u = u_1
  for (int k = lane; k < n; k += 32) ut[k] = tmp[k + n * k];
  for (int c = lane; c < nc; c += 32) {
    double sv = 0.0;
    if (c < n) {
      for (int a = 0; a < n; ++a) sv += T->D[c * n + a] * tmp[a + n * c];
    } else {
      const double* lv = (c == n) ? T->l1 : T->l0;
      for (int b = 0; b < n; ++b) {
        double t = 0.0;
        for (int a = 0; a < n; ++a) t += lv[a] * tmp[a + n * b];
        sv += lv[b] * t;
      }
    }
    zu[c] = sv;
  }
  __syncwarp();
  double* kc = A.kco + (size_t)e * (2 * nc * n + nn);
  for (int q = lane; q < 2 * nc * n + nn; q += 32) {
    double v = 0.0;
    if (q < nc * n) {                       // Cx of D1: x-lines by y index j
      const int c = q / n, j = q % n;
      for (int k = 0; k < n; ++k) v += ut[k] * Cx3[(size_t)c * nn + j + n * k];
    } else if (q < 2 * nc * n) {            // Cy of D1: y-lines by x index i
      const int c = (q - nc * n) / n, i = (q - nc * n) % n;
      for (int k = 0; k < n; ++k) v += ut[k] * Cy3[(size_t)c * nn + i + n * k];
    } else {                                // diagonal: mass and Y1^T u_1
      const int d = q - 2 * nc * n, i = d % n, j = d / n;
      for (int k = 0; k < n; ++k) v += ut[k] * h3 * T->w[i] * T->w[j] * T->w[k];
      for (int c = 0; c < nc; ++c) v += Cz3[(size_t)c * nn + d] * zu[c];
    }
    kc[q] = irs * v;
  }
  // ---- 5. A1^-1 (Gauss-Jordan, one warp)
  for (int q = lane; q < 2 * nn; q += 32) {
    const int c = q / n, rr = q % n;
    aug[q] = (c < n) ? rs * tmp[rr + n * c] : ((rr == c - n) ? 1.0 : 0.0);
  }
  __syncwarp();
  const double na = norm1_warp(aug, n);
  const bool sing = warp_gauss_jordan(aug, n, fac);
  const double ni = norm1_warp(aug + nn, n);
  for (int q = lane; q < nn; q += 32) A.Azi[e * nn + q] = aug[nn + q];
  if (lane == 0) {
    A.sigz[e] = s1;
    const double cnd = na * ni;
    int zf = 0;
    if (!conv) zf |= 1;
    if (sing || !(cnd < 1e14)) zf |= 2;
    A.zflags[e] = zf;
    if (zf & 1) atomicAdd(&A.st->z_unconverged, 1);
    if (zf & 2) atomicAdd(&A.st->build_singular, 1);
    if (cnd < 1e300) atomic_max_double(&A.st->max_cond_z, cnd);
  }
}

cudaError_t launch_build_3d(const tpp_ctx* c, cudaStream_t s) {
  const int n = c->n;
  Stage1Args a;
  a.T = c->p<Tables>(c->L.tables);
  a.n = n;
  a.rz = c->rz;
  a.Jmax = s1_jmax(n);
  a.E = c->E;
  a.h = c->prob.h;
  a.cx = c->p<double>(c->L.cx);
  a.cy = c->p<double>(c->L.cy);
  a.cz = c->p<double>(c->L.cz);
  a.fa = c->p<double>(c->L.fa);
  a.Zd = c->p<double>(c->L.zd);
  a.Rz = c->p<double>(c->L.rz);
  a.scr = c->p<double>(c->L.s1scr);
  a.kco = c->p<double>(c->L.kco);
  a.Az = c->p<double>(c->L.fAz);
  a.Azi = c->p<double>(c->L.fAzi);
  a.sigz = c->p<double>(c->L.sigz);
  a.zflags = c->p<int32_t>(c->L.zflags);
  a.st = c->p<DevStatus>(c->L.status);
  const int warps = 4;
  const size_t smem = (size_t)warps * (2 * n * n + n + 40 + 520) * sizeof(double);
  k_stage1_3d<<<(unsigned)((c->E + warps - 1) / warps), warps * 32, smem, s>>>(a);
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_ksvd_pipeline(c, s, nullptr);
}

}  // namespace tpp
