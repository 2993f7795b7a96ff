// Full multi-component blocks of the Euler systems (Sec. 5.3, Sec. 5.6).  In 2D: the
// Kronecker approximation A_1 (x) B_1 + A_2 (x) B_2 of each element's whole
// n_c n^2 x n_c n^2 Jacobian block, A_k of size n_c n x n_c n acting on the
// (component, y) index a = c n + j, B_k of size n x n acting on x.  In 3D: the nested
// form of Sec. 4.3 with the component on the z factor (second part of this file).  In
// both: the exact full-block Jacobi comparator (J_full).
//
// Rearranged block.  With the collocated coefficients of the coupled operator
// (k_system.cu) the block is a sum of 2n + 2 Kronecker terms alpha_t (x) beta_t:
//   t <  n      x volume:   beta_t[i][i'] = d(i', t) D[t][i],
//                           alpha_t[a][a'] = d(j, j') cx[c][c'](t, j)
//   t = n + s   x-diagonal: beta_t = e_s e_s^T,
//               alpha_t[a][a'] = d(c,c') d(j,j') h^2 w_s w_j + D[j'][j] cy[c][c'](s, j')
//                              + l0_j l0_j' fo[-y][c][c'](s) + l1_j l1_j' fo[+y][c][c'](s)
//   t = 2n, 2n+1  x faces:  beta = l0 l0^T, l1 l1^T, alpha[a][a'] = d(j, j') fo[-x / +x][c][c'](j)
// so the rearrangement R = sum_t vec(alpha_t) vec(beta_t)^T has rank <= 2n + 2.  The
// beta_t do not depend on the element: beta = Q_B R_B once per context (CGS2 with
// dependent columns dropped), and the top-2 singular triplets of R are those of
// alpha R_B^T, found from the eigenvectors of the small Gram matrix
// G = R_B (alpha^T alpha) R_B^T (cyclic Jacobi, one CTA per element).  The
// singular values are well separated for these blocks (sigma_2 / sigma_1 of 0.3 to
// 0.95, sigma_3 / sigma_1 below 0.25), so the Gram form loses no digits that matter.
//
// Inverse (Sec. 4.2 with the Schur form on the small side).  With C = B_1^-1 B_2 =
// Q T Q^T (real Schur form), the system A_1 X B_1^T + A_2 X B_2^T = F (X, F of size
// m x n, m = n_c n) becomes, for Z = X Q and H = F B_1^-T Q,
//   A_1 Z + A_2 Z T^T = H,
// solved column by column from the last: (A_1 + T[k][k] A_2) z_k = h_k - A_2 sum_{l>k}
// T[k][l] z_l, a 2 m x 2 m coupled system for a 2 x 2 block of T.  The inverses of
// these shifted m x m (2 m x 2 m) systems are stored; X = Z Q^T.
#include <algorithm>
#include <cmath>

#include "tpp_internal.cuh"
#include "k_schur.cuh"

namespace tpp {

namespace {

constexpr int kNcFull = 4;          // 2D Euler: rho, rho u, rho v, rho E

__host__ __device__ inline int full_r(int n) { return 2 * n + 2; }

// in-place Gauss-Jordan inverse of the dm x dm row-major matrix M (shared memory) by the
// whole CTA, partial pivoting; fcol (dm doubles), red (blockDim / 32 doubles), perm (dm
// ints) are scratch.  Returns false if a pivot is zero or below 1e-300.
__device__ bool cta_gauss_jordan(double* M, int dm, double* fcol, double* red, int* perm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_piv;
  bool ok = true;
  for (int k = 0; k < dm; ++k) {
    // pivot search: largest |M[i][k]|, i >= k (lowest index among ties)
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < dm; i += nt) {
      const double v = fabs(M[i * dm + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    __syncthreads();
    if ((tid & 31) == 0) {
      red[tid >> 5] = best;
      reinterpret_cast<int*>(fcol)[tid >> 5] = bi;   // fcol is free until the elimination
    }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int ib = k;
      for (int w = 0; w < (nt >> 5); ++w) {
        const double v = red[w];
        const int iv = reinterpret_cast<int*>(fcol)[w];
        if (v > b || (v == b && iv < ib)) { b = v; ib = iv; }
      }
      s_piv = ib;
      perm[k] = ib;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != k)
      for (int j = tid; j < dm; j += nt) {
        const double t = M[k * dm + j];
        M[k * dm + j] = M[p * dm + j];
        M[p * dm + j] = t;
      }
    __syncthreads();
    const double pv = M[k * dm + k];
    if (!(fabs(pv) > 1e-300)) { ok = false; break; }       // uniform: every thread reads pv
    const double ip = 1.0 / pv;
    for (int i = tid; i < dm; i += nt) fcol[i] = (i == k) ? 0.0 : M[i * dm + k];
    __syncthreads();
    for (int j = tid; j < dm; j += nt) M[k * dm + j] = (j == k) ? ip : M[k * dm + j] * ip;
    __syncthreads();
    for (int q = tid; q < dm * dm; q += nt) {
      const int i = q / dm, j = q % dm;
      if (i == k) continue;
      const double f = fcol[i];
      M[q] = (j == k) ? -f * ip : M[q] - f * M[k * dm + j];
    }
    __syncthreads();
  }
  if (!ok) return false;
  for (int k = dm - 1; k >= 0; --k) {                       // undo the row interchanges
    const int p = perm[k];
    if (p != k)
      for (int i = tid; i < dm; i += nt) {
        const double t = M[i * dm + k];
        M[i * dm + k] = M[i * dm + p];
        M[i * dm + p] = t;
      }
    __syncthreads();
  }
  return true;
}

// column t of the element-independent basis: beta_t[i * n + i'] (see the file header)
__device__ __forceinline__ double beta_entry(const Tables* T, int n, int t, int i, int ip) {
  if (t < n) return (ip == t) ? T->D[t * n + i] : 0.0;
  if (t < 2 * n) return (i == t - n && ip == t - n) ? 1.0 : 0.0;
  if (t == 2 * n) return T->l0[i] * T->l0[ip];
  return T->l1[i] * T->l1[ip];
}

// beta = Q_B R_B: QB [rk][n^2] orthonormal columns, RB [r][r] row-major (rows < rk
// used), *rk the rank.  One CTA of 256 threads (n <= 16: one entry per thread).
__global__ void __launch_bounds__(256) k_full_basis(const Tables* T, int n, double* QB,
                                                    double* RB, int32_t* rk_out) {
  __shared__ double red[8];
  const int nn = n * n, r = full_r(n), tid = threadIdx.x;
  const int i = tid / n, ip = tid % n;
  int rk = 0;
  for (int q = tid; q < r * r; q += blockDim.x) RB[q] = 0.0;
  __syncthreads();
  for (int t = 0; t < r; ++t) {
    double v = (tid < nn) ? beta_entry(T, n, t, i, ip) : 0.0;
    const double n0 = sqrt(block_sum(v * v, red));
    for (int pass = 0; pass < 2; ++pass)
      for (int p = 0; p < rk; ++p) {
        const double qp = (tid < nn) ? QB[(size_t)p * nn + tid] : 0.0;
        const double cf = block_sum(v * qp, red);
        v -= cf * qp;
        if (tid == 0) RB[p * r + t] += cf;
      }
    const double nv = sqrt(block_sum(v * v, red));
    if (n0 > 0.0 && nv > 1e-10 * n0) {
      if (tid < nn) QB[(size_t)rk * nn + tid] = v / nv;
      if (tid == 0) RB[rk * r + t] = nv;
      ++rk;
    }
    __syncthreads();
  }
  if (tid == 0) *rk_out = rk;
}

struct FullArgs {
  const Tables* T;
  int n;
  int64_t E;
  double hd;                 // h^2 (collocated mass scale)
  const double* cx;          // [E][NC][NC][n^2] coupled volume coefficients (k_system.cu)
  const double* cy;
  const double* fo;          // [E][4][NC][NC][n] own-face coefficients
  const double* QB;
  const double* RB;
  const int32_t* rk;
  double* A;                 // [E][2][m][m] row-major
  double* B;                 // [E][2][n][n] row-major
  double* sig;               // [E][2]
  int32_t* flags;            // [E]
  DevStatus* st;
};

struct FullKsvdSmem {
  int tab, gx, dch, W, G, V, tmp, gam, red, rot, total, ch;
};

__host__ __device__ inline FullKsvdSmem full_ksvd_smem(int n) {
  const int nn = n * n, m = kNcFull * n, r = full_r(n);
  FullKsvdSmem s;
  int o = 0;
  s.tab = o; o += nn + 3 * n;
  s.gx = o; o += (n + 2) * kNcFull * kNcFull * n;
  const int chq = 8192 / (n * m);
  s.ch = chq < 1 ? 1 : (chq > m ? m : chq);
  s.dch = o; o += n * s.ch * m;
  s.W = o; o += r * r;
  s.G = o; o += r * r;
  s.V = o; o += r * r;
  s.tmp = o; o += r * r;
  s.gam = o; o += 2 * r;
  s.red = o; o += 8;
  s.rot = o; o += 2 * r;     // c, s per pair
  s.total = o;
  return s;
}

// alpha_{n+s}[a][a'] (the x-diagonal terms), a = c n + j, a' = c' n + j'
__device__ __forceinline__ double alpha_diag(const FullArgs& A, const double* Ds, const double* wl,
                                             int64_t e, int s, int a, int ap) {
  const int n = A.n, nn = n * n, NC = kNcFull;
  const int c = a / n, j = a % n, cp = ap / n, jp = ap % n;
  const int cc = c * NC + cp;
  double v = A.cy[((e * NC * NC) + cc) * nn + s + n * jp] * Ds[jp * n + j];
  const double* fe = A.fo + e * 4 * NC * NC * n;
  v += wl[n + j] * wl[n + jp] * fe[(2 * NC * NC + cc) * n + s];
  v += wl[2 * n + j] * wl[2 * n + jp] * fe[(3 * NC * NC + cc) * n + s];
  if (c == cp && j == jp) v += A.hd * wl[s] * wl[j];
  return v;
}

// one CTA (256 threads) per element: Gram matrix of the 2n + 2 terms, its top-2
// eigenpairs in the Q_B coordinates, and the factors
__global__ void __launch_bounds__(256) k_full_ksvd(FullArgs A) {
  extern __shared__ double sm[];
  const int n = A.n, nn = n * n, NC = kNcFull, m = NC * n, r = full_r(n);
  const int tid = threadIdx.x, nt = blockDim.x;
  const FullKsvdSmem L = full_ksvd_smem(n);
  const int64_t e = blockIdx.x;
  double* Ds = sm + L.tab;
  double* wl = Ds + nn;                       // w, l0, l1
  double* gx = sm + L.gx;                     // [n + 2][NC NC n]
  double* dch = sm + L.dch;                   // [n][ch][m]
  double* W = sm + L.W;
  double* G = sm + L.G;
  double* V = sm + L.V;
  double* Tm = sm + L.tmp;
  double* gam = sm + L.gam;
  double* red = sm + L.red;
  double* rot = sm + L.rot;
  const int rk = *A.rk;
  for (int q = tid; q < nn; q += nt) Ds[q] = A.T->D[q];
  for (int q = tid; q < n; q += nt) {
    wl[q] = A.T->w[q];
    wl[n + q] = A.T->l0[q];
    wl[2 * n + q] = A.T->l1[q];
  }
  const int gl = NC * NC * n;                 // length of an x-type coefficient vector
  const double* fe = A.fo + e * 4 * NC * NC * n;
  for (int q = tid; q < (n + 2) * gl; q += nt) {
    const int s = q / gl, k = q % gl, cc = k / n, j = k % n;
    gx[q] = (s < n) ? A.cx[(e * NC * NC + cc) * nn + s + n * j]
                    : fe[((s - n) * NC * NC + cc) * n + j];
  }
  __syncthreads();
  // index of x-set member s (0..n+1) among the 2n + 2 terms
  auto tx = [n](int s) { return s < n ? s : n + s; };
  // W = alpha^T alpha: x-x block
  for (int q = tid; q < (n + 2) * (n + 2); q += nt) {
    const int s = q / (n + 2), u = q % (n + 2);
    double acc = 0.0;
    for (int k = 0; k < gl; ++k) acc += gx[s * gl + k] * gx[u * gl + k];
    W[tx(s) * r + tx(u)] = acc;
  }
  // diagonal-diagonal and x-diagonal blocks, rows of alpha in chunks of L.ch
  double add = 0.0, axd0 = 0.0, axd1 = 0.0;
  const int ndd = n * n, nxd = (n + 2) * n;
  for (int a0 = 0; a0 < m; a0 += L.ch) {
    const int rows = min(L.ch, m - a0);
    __syncthreads();
    for (int q = tid; q < n * rows * m; q += nt) {
      const int s = q / (rows * m), rr = (q / m) % rows, ap = q % m;
      dch[(s * L.ch + rr) * m + ap] = alpha_diag(A, Ds, wl, e, s, a0 + rr, ap);
    }
    __syncthreads();
    if (tid < ndd) {
      const int s = tid / n, u = tid % n;
      const double* ps = dch + s * L.ch * m;
      const double* pu = dch + u * L.ch * m;
      for (int k = 0; k < rows * m; ++k) add += ps[k] * pu[k];
    }
    for (int h = 0; h < 2; ++h) {
      const int q = tid + h * nt;
      if (q >= nxd) continue;
      const int s = q / n, u = q % n;
      double acc = 0.0;
      for (int rr = 0; rr < rows; ++rr) {
        const int a = a0 + rr, c = a / n, j = a % n;
        for (int cp = 0; cp < NC; ++cp)
          acc += gx[s * gl + (c * NC + cp) * n + j] * dch[(u * L.ch + rr) * m + cp * n + j];
      }
      if (h == 0) axd0 += acc; else axd1 += acc;
    }
  }
  __syncthreads();
  if (tid < ndd) W[(n + tid / n) * r + n + tid % n] = add;
  for (int h = 0; h < 2; ++h) {
    const int q = tid + h * nt;
    if (q >= nxd) continue;
    const int s = q / n, u = q % n;
    const double v = h == 0 ? axd0 : axd1;
    W[tx(s) * r + n + u] = v;
    W[(n + u) * r + tx(s)] = v;
  }
  __syncthreads();
  // G = R_B W R_B^T (rk x rk)
  for (int q = tid; q < r * rk; q += nt) {
    const int t = q / rk, p = q % rk;
    double acc = 0.0;
    for (int u = 0; u < r; ++u) acc += W[t * r + u] * A.RB[p * r + u];
    Tm[t * rk + p] = acc;
  }
  __syncthreads();
  for (int q = tid; q < rk * rk; q += nt) {
    const int p = q / rk, p2 = q % rk;
    double acc = 0.0;
    for (int t = 0; t < r; ++t) acc += A.RB[p * r + t] * Tm[t * rk + p2];
    G[q] = acc;
    V[q] = (p == p2) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int q = tid; q < rk * rk; q += nt) {              // symmetrise
    const int p = q / rk, p2 = q % rk;
    if (p < p2) {
      const double v = 0.5 * (G[q] + G[p2 * rk + p]);
      G[q] = v;
      G[p2 * rk + p] = v;
    }
  }
  __syncthreads();
  // cyclic Jacobi, round-robin pairs (rp players, a dummy when rk is odd)
  const int rp = rk + (rk & 1), np = rp / 2;
  for (int sweep = 0; sweep < 40 && rk > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int q = tid; q < rk * rk; q += nt) {
      const double v = G[q] * G[q];
      tot += v;
      if (q / rk != q % rk) off += v;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > 1e-30 * tot)) break;
    for (int round = 0; round < rp - 1; ++round) {
      auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (rp - 1); };
      if (tid < np) {
        const int p = player(tid), q = player(rp - 1 - tid);
        double cs = 1.0, sn = 0.0;
        if (p < rk && q < rk) {
          const double apq = G[p * rk + q];
          if (fabs(apq) > 1e-300) {
            const double th = (G[q * rk + q] - G[p * rk + p]) / (2.0 * apq);
            const double t = (fabs(th) > 1e150) ? 0.5 / th
                                                : copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
            cs = 1.0 / sqrt(t * t + 1.0);
            sn = t * cs;
          }
        }
        rot[2 * tid] = cs;
        rot[2 * tid + 1] = sn;
      }
      __syncthreads();
      for (int q = tid; q < np * rk; q += nt) {             // rows p, q
        const int i = q / rk, k = q % rk;
        const int p = player(i), p2 = player(rp - 1 - i);
        if (p >= rk || p2 >= rk) continue;
        const double cs = rot[2 * i], sn = rot[2 * i + 1];
        const double gp = G[p * rk + k], gq = G[p2 * rk + k];
        G[p * rk + k] = cs * gp - sn * gq;
        G[p2 * rk + k] = sn * gp + cs * gq;
      }
      __syncthreads();
      for (int q = tid; q < np * rk; q += nt) {             // columns p, q (and V)
        const int i = q / rk, k = q % rk;
        const int p = player(i), p2 = player(rp - 1 - i);
        if (p >= rk || p2 >= rk) continue;
        const double cs = rot[2 * i], sn = rot[2 * i + 1];
        const double gp = G[k * rk + p], gq = G[k * rk + p2];
        G[k * rk + p] = cs * gp - sn * gq;
        G[k * rk + p2] = sn * gp + cs * gq;
        const double vp = V[k * rk + p], vq = V[k * rk + p2];
        V[k * rk + p] = cs * vp - sn * vq;
        V[k * rk + p2] = sn * vp + cs * vq;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // the two largest eigenvalues (thread 0), then gamma_k = R_B^T v_k
  __shared__ int s_idx[2];
  __shared__ double s_sig[2];
  if (tid == 0) {
    int i1 = -1, i2 = -1;
    for (int p = 0; p < rk; ++p) {
      const double v = G[p * rk + p];
      if (i1 < 0 || v > G[i1 * rk + i1]) { i2 = i1; i1 = p; }
      else if (i2 < 0 || v > G[i2 * rk + i2]) i2 = p;
    }
    s_idx[0] = i1;
    s_idx[1] = i2;
    s_sig[0] = (i1 >= 0) ? sqrt(fmax(G[i1 * rk + i1], 0.0)) : 0.0;
    s_sig[1] = (i2 >= 0) ? sqrt(fmax(G[i2 * rk + i2], 0.0)) : 0.0;
  }
  __syncthreads();
  for (int q = tid; q < 2 * r; q += nt) {
    const int k = q / r, t = q % r, col = s_idx[k];
    double acc = 0.0;
    if (col >= 0)
      for (int p = 0; p < rk; ++p) acc += A.RB[p * r + t] * V[p * rk + col];
    gam[q] = acc;
  }
  __syncthreads();
  // B_k = sqrt(s_k) Q_B v_k, A_k = alpha gamma_k / sqrt(s_k)
  for (int k = 0; k < 2; ++k) {
    const double sg = s_sig[k];
    const int col = s_idx[k];
    const double rs = sqrt(sg), irs = (sg > 0.0) ? 1.0 / rs : 0.0;
    double* Bk = A.B + (e * 2 + k) * nn;
    for (int q = tid; q < nn; q += nt) {
      double acc = 0.0;
      if (col >= 0 && sg > 0.0)
        for (int p = 0; p < rk; ++p) acc += A.QB[(size_t)p * nn + q] * V[p * rk + col];
      Bk[q] = rs * acc;
    }
    const double* g = gam + k * r;
    double* Ak = A.A + (e * 2 + k) * (int64_t)m * m;
    for (int q = tid; q < m * m; q += nt) {
      const int a = q / m, ap = q % m;
      double acc = 0.0;
      if (sg > 0.0) {
        if (a % n == ap % n) {
          const int j = a % n, cc = (a / n) * NC + ap / n;
          for (int s = 0; s < n + 2; ++s) acc += gx[s * gl + cc * n + j] * g[tx(s)];
        }
        for (int s = 0; s < n; ++s) acc += alpha_diag(A, Ds, wl, e, s, a, ap) * g[n + s];
      }
      Ak[q] = acc * irs;
    }
  }
  if (tid == 0) {
    A.sig[e * 2] = s_sig[0];
    A.sig[e * 2 + 1] = s_sig[1];
    int fl = 0;
    if (!(s_sig[0] > 0.0)) fl |= 8;
    if (!(s_sig[1] > 0.0)) {
      fl |= 2;
      atomicAdd(&A.st->build_rank1, 1);
    }
    A.flags[e] = fl;
  }
}


// one warp per element: B_1^-1 (Gauss-Jordan, partial pivoting), C = B_1^-1 B_2, its
// real Schur form C = Q T Q^T, and M_b = B_1^-T Q.  Outputs row-major n x n.
__global__ void __launch_bounds__(128) k_full_bside(int n, int64_t E, const double* B,
                                                    double* Tout, double* Qout, double* Mbout,
                                                    int32_t* flags, DevStatus* st) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nn = n * n, ld = ld_of(n);
  const int64_t e = (int64_t)blockIdx.x * 4 + w;
  if (e >= E) return;                                        // whole warp
  const int per = 2 * nn + 2 * n * ld + 2 * n + 8;
  double* Bi = sm + w * per;        // row-major, inverted in place
  double* B2 = Bi + nn;             // row-major
  double* C = B2 + nn;              // column-major, leading dimension ld
  double* Q = C + n * ld;
  double* fc = Q + n * ld;          // n
  double* vb = fc + n;              // n + 8
  __shared__ int perm_all[4][32];
  int* perm = perm_all[w];
  const double* B1g = B + (e * 2) * nn;
  for (int q = lane; q < nn; q += 32) {
    Bi[q] = B1g[q];
    B2[q] = B1g[nn + q];
  }
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < n && ok; ++k) {
    double best = -1.0;
    int bi = k;
    if (lane >= k && lane < n) { best = fabs(Bi[lane * n + k]); bi = lane; }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) perm[k] = bi;
    if (bi != k)
      for (int j = lane; j < n; j += 32) {
        const double t = Bi[k * n + j];
        Bi[k * n + j] = Bi[bi * n + j];
        Bi[bi * n + j] = t;
      }
    __syncwarp();
    const double pv = Bi[k * n + k];
    if (!(fabs(pv) > 1e-300)) { ok = false; break; }
    const double ip = 1.0 / pv;
    for (int i = lane; i < n; i += 32) fc[i] = (i == k) ? 0.0 : Bi[i * n + k];
    __syncwarp();
    for (int j = lane; j < n; j += 32) Bi[k * n + j] = (j == k) ? ip : Bi[k * n + j] * ip;
    __syncwarp();
    for (int q = lane; q < nn; q += 32) {
      const int i = q / n, j = q % n;
      if (i == k) continue;
      Bi[q] = (j == k) ? -fc[i] * ip : Bi[q] - fc[i] * Bi[k * n + j];
    }
    __syncwarp();
  }
  int fl = 0;
  if (ok) {
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k)
        for (int i = lane; i < n; i += 32) {
          const double t = Bi[i * n + k];
          Bi[i * n + k] = Bi[i * n + p];
          Bi[i * n + p] = t;
        }
      __syncwarp();
    }
    for (int q = lane; q < nn; q += 32) {
      const int r = q % n, c = q / n;
      double acc = 0.0;
      for (int l = 0; l < n; ++l) acc += Bi[r * n + l] * B2[l * n + c];
      C[r + ld * c] = acc;
    }
    __syncwarp();
    bool relaxed = false;
    if (!warp_real_schur(C, Q, n, ld, vb, &relaxed)) fl |= 4;
    if (relaxed) fl |= 16;
    __syncwarp();
    double* Te = Tout + e * nn;
    double* Qe = Qout + e * nn;
    double* Me = Mbout + e * nn;
    for (int q = lane; q < nn; q += 32) {
      const int r = q / n, c = q % n;
      Te[q] = C[r + ld * c];
      Qe[q] = Q[r + ld * c];
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc += Bi[i * n + r] * Q[i + ld * c];
      Me[q] = acc;
    }
  } else {
    fl |= 8;
  }
  if (lane == 0) {
    if (fl & 4) atomicAdd(&st->build_schur_fail, 1);
    if (fl & 8) atomicAdd(&st->build_singular, 1);
    if (fl & 16) atomicAdd(&st->build_schur_relaxed, 1);
    flags[e] |= fl;
  }
}

// one CTA per (element, column k of T): the inverse of A_1 + T[k][k] A_2 (m x m), or of
// the coupled 2 m x 2 m system of a 2 x 2 block starting at k, into slots k (and k + 1)
// of the element's 2 n m^2 doubles
__global__ void __launch_bounds__(256) k_full_shift(int n, int64_t E, const double* A,
                                                    const double* T, double* inv, int32_t* flags,
                                                    DevStatus* st) {
  extern __shared__ double sm[];
  const int m = kNcFull * n, nn = n * n;
  const int64_t e = blockIdx.x / n;
  const int k = blockIdx.x % n;
  const double* Te = T + e * nn;
  if (k > 0 && Te[k * n + k - 1] != 0.0) return;            // second column of a 2 x 2 block
  const int bs = (k + 1 < n && Te[(k + 1) * n + k] != 0.0) ? 2 : 1, dm = bs * m;
  double* M = sm;                      // dm x dm
  double* fcol = M + dm * dm;          // dm + 8
  double* red = fcol + dm + 8;         // 8
  int* perm = reinterpret_cast<int*>(red + 8);
  const double* A1 = A + e * 2 * (int64_t)m * m;
  const double* A2 = A1 + (int64_t)m * m;
  for (int q = threadIdx.x; q < dm * dm; q += blockDim.x) {
    const int R = q / dm, Cc = q % dm;
    const int p = R / m, a = R % m, pq = Cc / m, ap = Cc % m;
    double v = Te[(k + p) * n + (k + pq)] * A2[a * m + ap];
    if (p == pq) v += A1[a * m + ap];
    M[q] = v;
  }
  __syncthreads();
  const bool ok = cta_gauss_jordan(M, dm, fcol, red, perm);
  double* out = inv + e * 2 * (int64_t)n * m * m + (int64_t)k * 2 * m * m;
  for (int q = threadIdx.x; q < dm * dm; q += blockDim.x) out[q] = ok ? M[q] : 0.0;
  if (!ok && threadIdx.x == 0) {
    atomicOr(&flags[e], 8);
    atomicAdd(&st->build_singular, 1);
  }
}

struct FullApplyArgs {
  int n;
  int64_t E;
  const double* T;
  const double* Q;
  const double* Mb;
  const double* A;
  const double* inv;
  const double* b;
  double* x;
  const int32_t* skip;
};

// x = (A_1 (x) B_1 + A_2 (x) B_2)^-1 b, one CTA (256 threads) per element
__global__ void __launch_bounds__(256) k_full_apply(FullApplyArgs P) {
  if (P.skip && *P.skip) return;
  extern __shared__ double sm[];
  const int n = P.n, nn = n * n, m = kNcFull * n, mn = m * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int sub = tid & 3, rsl = tid >> 2, rows_per_pass = nt >> 2;
  const int64_t e = blockIdx.x;
  double* F = sm;                 // m x n: b, then H = F M_b
  double* H = F + mn;
  double* Z = H + mn;
  double* U = Z + mn;             // A_2 z_l
  double* A2 = U + mn;            // m x m
  double* Ts = A2 + m * m;
  double* Qs = Ts + nn;
  double* Ms = Qs + nn;
  double* rhs = Ms + nn;          // 2 m
  const double* A2g = P.A + (e * 2 + 1) * (int64_t)m * m;
  for (int q = tid; q < mn; q += nt) F[q] = P.b[e * mn + q];
  for (int q = tid; q < m * m; q += nt) A2[q] = A2g[q];
  for (int q = tid; q < nn; q += nt) {
    Ts[q] = P.T[e * nn + q];
    Qs[q] = P.Q[e * nn + q];
    Ms[q] = P.Mb[e * nn + q];
  }
  __syncthreads();
  for (int q = tid; q < mn; q += nt) {
    const int a = q / n, k = q % n;
    double acc = 0.0;
    for (int l = 0; l < n; ++l) acc += F[a * n + l] * Ms[l * n + k];
    H[q] = acc;
  }
  __syncthreads();
  const double* inv = P.inv + e * 2 * (int64_t)n * m * m;
  int k = n - 1;
  while (k >= 0) {
    const int k0 = (k > 0 && Ts[k * n + k - 1] != 0.0) ? k - 1 : k;
    const int bs = k - k0 + 1, dm = bs * m;
    for (int q = tid; q < dm; q += nt) {
      const int p = q / m, a = q % m, row = k0 + p;
      double v = H[a * n + row];
      for (int l = k + 1; l < n; ++l) v -= Ts[row * n + l] * U[a * n + l];
      rhs[q] = v;
    }
    __syncthreads();
    // matvecs with four threads per row (two shuffle-adds per row instead of five per
    // warp-split row: the FP64 pipe, not HBM, bounds this kernel)
    const double* G = inv + (int64_t)k0 * 2 * m * m;
    for (int r0 = 0; r0 < dm; r0 += rows_per_pass) {
      const int row = r0 + rsl;
      const bool ok = row < dm;
      double acc = 0.0;
      if (ok)
        for (int c = sub; c < dm; c += 4) acc += G[(int64_t)row * dm + c] * rhs[c];
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (ok && sub == 0) Z[(row % m) * n + k0 + row / m] = acc;
    }
    __syncthreads();
    for (int r0 = 0; r0 < dm; r0 += rows_per_pass) {
      const int row = r0 + rsl;
      const bool ok = row < dm;
      const int p = row / m, a = row % m;
      double acc = 0.0;
      if (ok)
        for (int c = sub; c < m; c += 4) acc += A2[a * m + c] * Z[c * n + k0 + p];
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (ok && sub == 0) U[a * n + k0 + p] = acc;
    }
    __syncthreads();
    k = k0 - 1;
  }
  for (int q = tid; q < mn; q += nt) {
    const int a = q / n, i = q % n;
    double acc = 0.0;
    for (int l = 0; l < n; ++l) acc += Z[a * n + l] * Qs[i * n + l];
    P.x[e * mn + q] = acc;
  }
}

// ---- 3D full blocks: the nested form A_1 (x) (B_1 (x) C_1 + B_2 (x) C_2) of Sec. 4.3
// with A_1 of size m = 5n on the (component, z) index a = c n + k, B_k on y, C_k on x.
// First stage (rank 1 in the a x (j, i) split): the block is sum_t alpha_t (x) beta_t over
// r1 = 3n^2 + 4n terms with element-independent beta_t (n^2 x n^2 on (j, i)):
//   t = i' + n j              x volume   beta[(j, i1)][(j, i')] = D[i'][i1]
//   t = n^2 + i + n j'        y volume   beta[(j1, i)][(j', i)] = D[j'][j1]
//   t = 2n^2 + i + n j        diagonal   beta = e_(j,i) e_(j,i)^T (mass, z volume, z faces)
//   t = 3n^2 + j + n f        x faces    beta[(j, i1)][(j, i2)] = l_f[i1] l_f[i2]
//   t = 3n^2 + 2n + i + n f   y faces    beta[(j1, i)][(j2, i)] = l_f[j1] l_f[j2]
// The top right singular vector lies in span(beta): v = sum_t mu_t beta_t and
// R^T R v = beta (alpha^T alpha) (beta^T beta) mu, so the power iteration runs on mu with
// the Gram matrix G_B = beta^T beta (once per context) and matrix-free alpha products.
// The second stage: D_1 = sum_t d_t beta_t is itself a sum of products of the 2n + 2 terms
// of the 2D basis (k_full_basis) on y and on x, D_1 = sum K[s][t] phi_s (x) phi_t, so its
// rank-2 KSVD is the SVD of the small core R_B K R_B^T (one-sided Jacobi).

__host__ __device__ inline int full3_r1(int n) { return 3 * n * n + 4 * n; }

// beta_t at row (j1, i1), column (j2, i2)
__device__ double beta3(const Tables* T, int n, int t, int j1, int i1, int j2, int i2) {
  const int nn = n * n;
  if (t < nn) {
    const int ip = t % n, j = t / n;
    return (j1 == j && j2 == j && i2 == ip) ? T->D[ip * n + i1] : 0.0;
  }
  if (t < 2 * nn) {
    const int u = t - nn, i = u % n, jp = u / n;
    return (i1 == i && i2 == i && j2 == jp) ? T->D[jp * n + j1] : 0.0;
  }
  if (t < 3 * nn) {
    const int u = t - 2 * nn, i = u % n, j = u / n;
    return (j1 == j && i1 == i && j2 == j && i2 == i) ? 1.0 : 0.0;
  }
  const int u = t - 3 * nn;
  if (u < 2 * n) {
    const int j = u % n;
    const double* l = (u / n) ? T->l1 : T->l0;
    return (j1 == j && j2 == j) ? l[i1] * l[i2] : 0.0;
  }
  const int v = u - 2 * n, i = v % n;
  const double* l = (v / n) ? T->l1 : T->l0;
  return (i1 == i && i2 == i) ? l[j1] * l[j2] : 0.0;
}

// G_B[s][t] = <beta_s, beta_t>: the sum over the (at most n^2) nonzeros of beta_s
__global__ void k_full3_gram(const Tables* T, int n, double* GB) {
  const int r1 = full3_r1(n), nn = n * n;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= r1 * r1) return;
  const int s = q / r1, t = q % r1;
  double acc = 0.0;
  if (s < nn) {
    const int ip = s % n, j = s / n;
    for (int i1 = 0; i1 < n; ++i1) acc += T->D[ip * n + i1] * beta3(T, n, t, j, i1, j, ip);
  } else if (s < 2 * nn) {
    const int u = s - nn, i = u % n, jp = u / n;
    for (int j1 = 0; j1 < n; ++j1) acc += T->D[jp * n + j1] * beta3(T, n, t, j1, i, jp, i);
  } else if (s < 3 * nn) {
    const int u = s - 2 * nn, i = u % n, j = u / n;
    acc = beta3(T, n, t, j, i, j, i);
  } else if (s < 3 * nn + 2 * n) {
    const int u = s - 3 * nn, j = u % n;
    const double* l = (u / n) ? T->l1 : T->l0;
    for (int i1 = 0; i1 < n; ++i1)
      for (int i2 = 0; i2 < n; ++i2) acc += l[i1] * l[i2] * beta3(T, n, t, j, i1, j, i2);
  } else {
    const int v = s - 3 * nn - 2 * n, i = v % n;
    const double* l = (v / n) ? T->l1 : T->l0;
    for (int j1 = 0; j1 < n; ++j1)
      for (int j2 = 0; j2 < n; ++j2) acc += l[j1] * l[j2] * beta3(T, n, t, j1, i, j2, i);
  }
  GB[q] = acc;
}

struct Full3Args {
  const Tables* T;
  int n;
  int64_t E;
  double h3;
  const double* cx;          // [E][5][5][n^3] coupled volume coefficients (k_system.cu)
  const double* cy;
  const double* cz;
  const double* fo;          // [E][6][5][5][n^2] own-face coefficients
  const double* GB;          // [r1][r1]
  const double* QB;          // 2D basis (k_full_basis)
  const double* RB;
  const int32_t* rk;
  double* A;                 // [E][m][m] first-stage factor A_1, row-major
  double* Ainv;              // [E][m][m] its inverse
  double* sig;               // [E][2]: sigma_1 of the first stage, power iterations
  int32_t* flags;            // [E] bit0 not converged, bit3 A_1 singular
  double* A1;                // second-stage factors into the small-block context's arrays
  double* B1;                // ([E][n*n] column-major, B_k on y as "A", C_k on x as "B")
  double* A2;
  double* B2;
  double* sigma;             // [E][2] second-stage singular values
  DevStatus* st;
};

// alpha_t[(c, k)][(c', k')] of element e (see the 3D header above)
__device__ double alpha3(const Full3Args& P, const double* wl, int64_t e, int t, int c, int k,
                         int cp, int kp) {
  constexpr int NC = 5;
  const int n = P.n, nn = n * n, n3 = nn * n, cc = c * NC + cp;
  const int64_t vb = (e * NC * NC + cc) * (int64_t)n3;
  const double* fe = P.fo + e * 6 * NC * NC * nn;
  if (t < nn) return (k == kp) ? P.cx[vb + (t % n) + n * (t / n) + nn * k] : 0.0;
  if (t < 2 * nn) {
    const int u = t - nn;
    return (k == kp) ? P.cy[vb + (u % n) + n * (u / n) + nn * k] : 0.0;
  }
  if (t < 3 * nn) {
    const int u = t - 2 * nn, i = u % n, j = u / n;
    double v = P.T->D[kp * n + k] * P.cz[vb + i + n * j + nn * kp];
    v += wl[n + k] * wl[n + kp] * fe[(4 * NC * NC + cc) * nn + u];
    v += wl[2 * n + k] * wl[2 * n + kp] * fe[(5 * NC * NC + cc) * nn + u];
    if (c == cp && k == kp) v += P.h3 * wl[i] * wl[j] * wl[k];
    return v;
  }
  if (k != kp) return 0.0;
  const int u = t - 3 * nn;
  if (u < 2 * n) return fe[((u / n) * NC * NC + cc) * nn + (u % n) + n * k];
  const int v = u - 2 * n;
  return fe[((2 + v / n) * NC * NC + cc) * nn + (v % n) + n * k];
}

struct Full3Smem {
  int tab, mu, y, z, u, K, W, V, fc, total;
};

__host__ __device__ inline Full3Smem full3_smem(int n) {
  const int m = 5 * n, r1 = full3_r1(n), r = full_r(n);
  Full3Smem s;
  int o = 0;
  s.tab = o; o += n * n + 3 * n;
  s.mu = o; o += r1;
  s.y = o; o += r1;
  s.z = o; o += r1;
  s.u = o; o += m * m;
  s.K = o; o += r * r;
  s.W = o; o += r * r;
  s.V = o; o += r * r;
  s.fc = o; o += m + 16 + (m + 1) / 2 + 1;   // Gauss-Jordan scratch (fcol, red, perm)
  s.total = o;
  return s;
}

// one CTA (256 threads) per element: first stage by power iteration, the second-stage
// factors, and A_1^-1
__global__ void __launch_bounds__(256) k_full3_build(Full3Args P) {
  extern __shared__ double sm[];
  constexpr int NC = 5;
  const int n = P.n, nn = n * n, m = NC * n, mm = m * m, r1 = full3_r1(n), r = full_r(n);
  const int tid = threadIdx.x, nt = blockDim.x;
  const Full3Smem L = full3_smem(n);
  const int64_t e = blockIdx.x;
  double* wl = sm + L.tab + nn;         // w, l0, l1
  double* mu = sm + L.mu;
  double* y = sm + L.y;
  double* z = sm + L.z;
  double* u = sm + L.u;
  double* K = sm + L.K;
  double* W = sm + L.W;
  double* V = sm + L.V;
  double* red = sm + L.fc + m + 8;      // 8 doubles inside the Gauss-Jordan scratch
  __shared__ double s_val[4];
  __shared__ double s_red[16];
  for (int q = tid; q < n; q += nt) {
    wl[q] = P.T->w[q];
    wl[n + q] = P.T->l0[q];
    wl[2 * n + q] = P.T->l1[q];
  }
  for (int q = tid; q < r1; q += nt) {  // start: the mass direction
    const int u2 = q - 2 * nn;
    mu[q] = (u2 >= 0 && u2 < nn) ? P.T->w[u2 % n] * P.T->w[u2 / n] : 0.0;
  }
  __syncthreads();
  // y = G_B mu, vv = mu . y, u = alpha y, uu = |u|^2
  auto forward = [&]() {
    for (int s = tid; s < r1; s += nt) {
      double acc = 0.0;
      for (int t = 0; t < r1; ++t) acc += P.GB[(size_t)t * r1 + s] * mu[t];   // symmetric
      y[s] = acc;
    }
    __syncthreads();
    for (int q = tid; q < mm; q += nt) {
      const int a = q / m, ap = q % m, c = a / n, k = a % n, cp = ap / n, kp = ap % n;
      double acc = 0.0;
      for (int t = 2 * nn; t < 3 * nn; ++t) acc += alpha3(P, wl, e, t, c, k, cp, kp) * y[t];
      if (k == kp) {
        for (int t = 0; t < 2 * nn; ++t) acc += alpha3(P, wl, e, t, c, k, cp, kp) * y[t];
        for (int t = 3 * nn; t < r1; ++t) acc += alpha3(P, wl, e, t, c, k, cp, kp) * y[t];
      }
      u[q] = acc;
    }
    double pv = 0.0, pu = 0.0;
    for (int s = tid; s < r1; s += nt) pv += mu[s] * y[s];
    for (int q = tid; q < mm; q += nt) pu += u[q] * u[q];
    const double vv = block_sum(pv, red);
    const double uu = block_sum(pu, red);
    if (tid == 0) {
      s_val[0] = vv;
      s_val[1] = uu;
    }
    __syncthreads();
  };
  forward();
  int it = 0;
  bool conv = false;
  for (; it < 500 && !conv; ++it) {
    const double vv = s_val[0], uu = s_val[1];
    if (!(vv > 0.0) || !(uu > 0.0)) break;
    const double lam = uu / vv;
    // z = alpha^T u
    for (int t = tid; t < r1; t += nt) {
      double acc = 0.0;
      if (t >= 2 * nn && t < 3 * nn) {
        for (int q = 0; q < mm; ++q) {
          const int a = q / m, ap = q % m;
          acc += alpha3(P, wl, e, t, a / n, a % n, ap / n, ap % n) * u[q];
        }
      } else {
        for (int c = 0; c < NC; ++c)
          for (int cp = 0; cp < NC; ++cp)
            for (int k = 0; k < n; ++k)
              acc += alpha3(P, wl, e, t, c, k, cp, k) * u[(c * n + k) * m + cp * n + k];
      }
      z[t] = acc / lam;
    }
    __syncthreads();
    double pd = 0.0, pm = 0.0;
    for (int t = tid; t < r1; t += nt) {
      pd = fmax(pd, fabs(z[t] - mu[t]));
      pm = fmax(pm, fabs(z[t]));
      mu[t] = z[t];
    }
    for (int o = 16; o > 0; o >>= 1) {
      pd = fmax(pd, __shfl_xor_sync(0xffffffffu, pd, o));
      pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, o));
    }
    __syncthreads();
    if ((tid & 31) == 0) {
      s_red[tid >> 5] = pd;
      s_red[8 + (tid >> 5)] = pm;
    }
    __syncthreads();
    double dmax = 0.0, mmax = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) {
      dmax = fmax(dmax, s_red[w]);
      mmax = fmax(mmax, s_red[8 + w]);
    }
    conv = dmax <= 1e-14 * mmax;
    __syncthreads();
    forward();
  }
  const double vv = s_val[0], uu = s_val[1];
  const double sig1 = (vv > 0.0) ? sqrt(uu / vv) : 0.0;
  const double sa = (sig1 > 0.0) ? 1.0 / sqrt(sig1 * vv) : 0.0;    // A_1 = u / sqrt(sig1 vv)
  const double sd = (vv > 0.0) ? sqrt(sig1 / vv) : 0.0;            // D_1 = sd sum mu_t beta_t
  for (int q = tid; q < mm; q += nt) {
    u[q] *= sa;
    P.A[e * mm + q] = u[q];
  }
  // K[s][t]: D_1 in the products of the 2D basis (s on y, t on x)
  for (int q = tid; q < r * r; q += nt) K[q] = 0.0;
  __syncthreads();
  if (tid == 0) {
    for (int t = 0; t < r1; ++t) {
      const double d = sd * mu[t];
      int row, col;
      if (t < nn) { row = n + t / n; col = t % n; }                         // x volume
      else if (t < 2 * nn) { row = (t - nn) / n; col = n + (t - nn) % n; }  // y volume
      else if (t < 3 * nn) { row = n + (t - 2 * nn) / n; col = n + (t - 2 * nn) % n; }
      else if (t < 3 * nn + 2 * n) { const int v = t - 3 * nn; row = n + v % n; col = 2 * n + v / n; }
      else { const int v = t - 3 * nn - 2 * n; row = 2 * n + v / n; col = n + v % n; }
      K[row * r + col] += d;
    }
  }
  __syncthreads();
  // core W = R_B K R_B^T (rk x rk), via V = K R_B^T
  const int rk = *P.rk;
  for (int q = tid; q < r * rk; q += nt) {
    const int s = q / rk, p = q % rk;
    double acc = 0.0;
    for (int t = 0; t < r; ++t) acc += K[s * r + t] * P.RB[p * r + t];
    V[s * rk + p] = acc;
  }
  __syncthreads();
  for (int q = tid; q < rk * rk; q += nt) {
    const int p = q / rk, p2 = q % rk;
    double acc = 0.0;
    for (int s = 0; s < r; ++s) acc += P.RB[p * r + s] * V[s * rk + p2];
    W[q] = acc;
  }
  __syncthreads();
  for (int q = tid; q < rk * rk; q += nt) V[q] = (q / rk == q % rk) ? 1.0 : 0.0;
  __syncthreads();
  // one-sided Jacobi: W V = U S, round-robin column pairs, one thread per pair
  const int rp = rk + (rk & 1), np = rp / 2;
  for (int sweep = 0; sweep < 40 && rk > 1; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < rp - 1; ++round) {
      if (tid < np) {
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (rp - 1); };
        const int p = player(tid), q2 = player(rp - 1 - tid);
        if (p < rk && q2 < rk) {
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int i = 0; i < rk; ++i) {
            const double wp = W[i * rk + p], wq = W[i * rk + q2];
            al += wp * wp;
            be += wq * wq;
            ga += wp * wq;
          }
          if (fabs(ga) > 1e-15 * sqrt(al * be) && fabs(ga) > 1e-300) {
            rotated = 1;
            const double ze = (be - al) / (2.0 * ga);
            const double t = (fabs(ze) > 1e150) ? 0.5 / ze
                                                : copysign(1.0, ze) / (fabs(ze) + sqrt(ze * ze + 1.0));
            const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
            for (int i = 0; i < rk; ++i) {
              const double wp = W[i * rk + p], wq = W[i * rk + q2];
              W[i * rk + p] = cs * wp - sn * wq;
              W[i * rk + q2] = sn * wp + cs * wq;
              const double vp = V[i * rk + p], vq = V[i * rk + q2];
              V[i * rk + p] = cs * vp - sn * vq;
              V[i * rk + q2] = sn * vp + cs * vq;
            }
          }
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  // the two largest column norms
  __shared__ int s_idx[2];
  __shared__ double s_sv[2];
  if (tid == 0) {
    int i1 = -1, i2 = -1;
    double n1 = -1.0, n2 = -1.0;
    for (int p = 0; p < rk; ++p) {
      double nr = 0.0;
      for (int i = 0; i < rk; ++i) nr += W[i * rk + p] * W[i * rk + p];
      if (nr > n1) { n2 = n1; i2 = i1; n1 = nr; i1 = p; }
      else if (nr > n2) { n2 = nr; i2 = p; }
    }
    s_idx[0] = i1;
    s_idx[1] = i2;
    s_sv[0] = (i1 >= 0) ? sqrt(n1) : 0.0;
    s_sv[1] = (i2 >= 0) ? sqrt(n2) : 0.0;
  }
  __syncthreads();
  // B_k (y) = sqrt(s_k) Q_B u_k with u_k = W[:, col] / s_k; C_k (x) = sqrt(s_k) Q_B V[:, col]
  for (int k2 = 0; k2 < 2; ++k2) {
    const int col = s_idx[k2];
    const double sv = s_sv[k2];
    const double rs = sqrt(sv), irs = (sv > 0.0) ? 1.0 / rs : 0.0;
    double* By = (k2 == 0 ? P.A1 : P.A2) + e * nn;
    double* Cx = (k2 == 0 ? P.B1 : P.B2) + e * nn;
    for (int q = tid; q < nn; q += nt) {
      double ay = 0.0, ax = 0.0;
      if (col >= 0 && sv > 0.0)
        for (int p = 0; p < rk; ++p) {
          ay += P.QB[(size_t)p * nn + q] * W[p * rk + col];
          ax += P.QB[(size_t)p * nn + q] * V[p * rk + col];
        }
      const int rr = q / n, cl = q % n;             // row-major [rr][cl] -> column-major
      By[rr + n * cl] = ay * irs;                   // sqrt(s) u = W[:, col] / sqrt(s)
      Cx[rr + n * cl] = ax * rs;
    }
    if (tid == 0) P.sigma[e * 2 + k2] = sv;
  }
  __syncthreads();
  // A_1^-1 (Gauss-Jordan in the u buffer)
  const bool ok = cta_gauss_jordan(u, m, sm + L.fc, red,
                                   reinterpret_cast<int*>(sm + L.fc + m + 16));
  for (int q = tid; q < mm; q += nt) P.Ainv[e * mm + q] = ok ? u[q] : 0.0;
  if (tid == 0) {
    P.sig[e * 2] = sig1;
    P.sig[e * 2 + 1] = (double)it;
    int fl = 0;
    if (!conv) {
      fl |= 1;
      atomicAdd(&P.st->z_unconverged, 1);
    }
    if (!ok) {
      fl |= 8;
      atomicAdd(&P.st->build_singular, 1);
    }
    P.flags[e] = fl;
  }
}

// x = (A_1^-1 (x) I) b along the (component, z) index, one CTA per element
__global__ void __launch_bounds__(256) k_full3_apply_z(int n, const double* Ainv, const double* b,
                                                       double* x, const int32_t* skip) {
  if (skip && *skip) return;
  extern __shared__ double sm[];
  const int m = 5 * n, nn = n * n, mm = m * m;
  const int64_t e = blockIdx.x;
  double* Ai = sm;
  double* bs = sm + mm;
  for (int q = threadIdx.x; q < mm; q += blockDim.x) Ai[q] = Ainv[e * mm + q];
  for (int q = threadIdx.x; q < m * nn; q += blockDim.x) bs[q] = b[e * m * nn + q];
  __syncthreads();
  for (int q = threadIdx.x; q < m * nn; q += blockDim.x) {
    const int a = q / nn, qq = q % nn;
    double acc = 0.0;
    for (int ap = 0; ap < m; ++ap) acc += Ai[a * m + ap] * bs[ap * nn + qq];
    x[e * m * nn + q] = acc;
  }
}

// the whole 3D n_c n^3 x n_c n^3 block (n_c = 5, node (c, k, j, i)), row-major: in each
// direction d the volume term D[a'][a] cd[c][c'](node at a') and the two own-face terms,
// the other two node coordinates equal
__global__ void k_full_bj_assemble_3d(const Tables* T, int n, double hd, const double* cx,
                                      const double* cy, const double* cz, const double* fo,
                                      double* LU) {
  constexpr int NC = 5;
  const int nn = n * n, n3 = nn * n, nb = NC * n3;
  const int64_t e = blockIdx.x;
  const double* fe = fo + e * 6 * NC * NC * nn;
  const double* cd[3] = {cx, cy, cz};
  double* Ae = LU + e * (int64_t)nb * nb;
  for (int64_t q = threadIdx.x; q < (int64_t)nb * nb; q += blockDim.x) {
    const int row = (int)(q / nb), col = (int)(q % nb);
    const int c = row / n3, cp = col / n3, rn = row % n3, cn = col % n3;
    const int r3[3] = {rn % n, (rn / n) % n, rn / nn};
    const int c3[3] = {cn % n, (cn / n) % n, cn / nn};
    const int cc = c * NC + cp;
    double v = 0.0;
    if (row == col) v += hd * T->w[r3[0]] * T->w[r3[1]] * T->w[r3[2]];
    for (int d = 0; d < 3; ++d) {
      const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
      if (r3[o1] != c3[o1] || r3[o2] != c3[o2]) continue;
      const int a = r3[d], ap = c3[d];
      v += T->D[ap * n + a] * cd[d][(e * NC * NC + cc) * (int64_t)n3 + cn];
      const int lo = (d == 0) ? 1 : 0, hi = (d == 2) ? 1 : 2;
      const int t = r3[lo] + n * r3[hi];
      v += T->l0[a] * T->l0[ap] * fe[((2 * d) * NC * NC + cc) * nn + t];
      v += T->l1[a] * T->l1[ap] * fe[((2 * d + 1) * NC * NC + cc) * nn + t];
    }
    Ae[q] = v;
  }
}

// the whole n_c n^2 x n_c n^2 block of element e, row-major, for exact block Jacobi
__global__ void k_full_bj_assemble(const Tables* T, int n, double hd, const double* cx,
                                   const double* cy, const double* fo, double* LU) {
  const int nn = n * n, NC = kNcFull, nb = NC * nn;
  const int64_t e = blockIdx.x;
  const double* fe = fo + e * 4 * NC * NC * n;
  double* Ae = LU + e * (int64_t)nb * nb;
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int row = q / nb, col = q % nb;
    const int c = row / nn, j = (row / n) % n, i = row % n;
    const int cp = col / nn, jp = (col / n) % n, ip = col % n;
    const int cc = c * NC + cp;
    double v = 0.0;
    if (c == cp && j == jp && i == ip) v += hd * T->w[i] * T->w[j];
    if (j == jp) {
      v += T->D[ip * n + i] * cx[(e * NC * NC + cc) * nn + ip + n * j];
      v += T->l0[i] * T->l0[ip] * fe[(0 * NC * NC + cc) * n + j];
      v += T->l1[i] * T->l1[ip] * fe[(1 * NC * NC + cc) * n + j];
    }
    if (i == ip) {
      v += T->D[jp * n + j] * cy[(e * NC * NC + cc) * nn + i + n * jp];
      v += T->l0[j] * T->l0[jp] * fe[(2 * NC * NC + cc) * n + i];
      v += T->l1[j] * T->l1[jp] * fe[(3 * NC * NC + cc) * n + i];
    }
    Ae[q] = v;
  }
}

}  // namespace

}  // namespace tpp

namespace tpp {

size_t full_layout(size_t base, int dim, int n, int64_t E, bool bj, FullOffsets* out) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t nn = (size_t)n * n, m = (size_t)kNcFull * n, r = (size_t)full_r(n);
  const size_t Ez = (size_t)E;
  FullOffsets L;
  size_t o = al(base);
  if (dim == 3) {                 // n_c = 5: A_1 of size 5n, blocks of 5 n^3
    const size_t m3 = 5 * (size_t)n, r1 = (size_t)full3_r1(n), nb = 5 * nn * (size_t)n;
    L.QB = o; o += al(nn * r * 8);
    L.RB = o; o += al(r * r * 8);
    L.rk = o; o += 256;
    L.GB = o; o += al(r1 * r1 * 8);
    L.A = o; o += al(Ez * m3 * m3 * 8);
    L.inv = o; o += al(Ez * m3 * m3 * 8);
    L.sig = o; o += al(Ez * 2 * 8);
    L.flags = o; o += al(Ez * 4);
    L.lu = bj ? o : 0; o += bj ? al(Ez * nb * nb * 8) : 0;
    L.piv = bj ? o : 0; o += bj ? al(Ez * nb * 4) : 0;
    L.total = o;
    if (out) *out = L;
    return o;
  }
  const size_t nb = (size_t)kNcFull * nn;
  L.QB = o; o += al(nn * r * 8);
  L.RB = o; o += al(r * r * 8);
  L.rk = o; o += 256;
  L.A = o; o += al(Ez * 2 * m * m * 8);
  L.B = o; o += al(Ez * 2 * nn * 8);
  L.sig = o; o += al(Ez * 2 * 8);
  L.T = o; o += al(Ez * nn * 8);
  L.Q = o; o += al(Ez * nn * 8);
  L.Mb = o; o += al(Ez * nn * 8);
  L.inv = o; o += al(Ez * 2 * n * m * m * 8);
  L.flags = o; o += al(Ez * 4);
  L.lu = bj ? o : 0; o += bj ? al(Ez * nb * nb * 8) : 0;
  L.piv = bj ? o : 0; o += bj ? al(Ez * nb * 4) : 0;
  L.total = o;
  if (out) *out = L;
  return o;
}

cudaError_t launch_full_basis(const tpp_ctx* c, cudaStream_t s) {
  k_full_basis<<<1, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->p<double>(c->fb.QB),
                                 c->p<double>(c->fb.RB), c->p<int32_t>(c->fb.rk));
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || c->dim != 3) return err;
  const int r1 = full3_r1(c->n);
  k_full3_gram<<<(unsigned)((r1 * r1 + 255) / 256), 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n,
                                                                 c->p<double>(c->fb.GB));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_full3_build(const tpp_ctx* c, cudaStream_t s) {
  Full3Args P;
  P.T = c->p<Tables>(c->L.tables);
  P.n = c->n;
  P.E = c->sys_E;
  P.h3 = c->prob.h * c->prob.h * c->prob.h;
  P.cx = c->p<double>(c->sys_cx);
  P.cy = c->p<double>(c->sys_cy);
  P.cz = c->p<double>(c->sys_cz);
  P.fo = c->p<double>(c->sys_fo);
  P.GB = c->p<double>(c->fb.GB);
  P.QB = c->p<double>(c->fb.QB);
  P.RB = c->p<double>(c->fb.RB);
  P.rk = c->p<int32_t>(c->fb.rk);
  P.A = c->p<double>(c->fb.A);
  P.Ainv = c->p<double>(c->fb.inv);
  P.sig = c->p<double>(c->fb.sig);
  P.flags = c->p<int32_t>(c->fb.flags);
  P.A1 = c->p<double>(c->L.fA1);
  P.B1 = c->p<double>(c->L.fB1);
  P.A2 = c->p<double>(c->L.fA2);
  P.B2 = c->p<double>(c->L.fB2);
  P.sigma = c->p<double>(c->L.sigma);
  P.st = c->p<DevStatus>(c->L.status);
  const size_t smem = (size_t)full3_smem(c->n).total * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(k_full3_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  k_full3_build<<<(unsigned)c->sys_E, 256, smem, s>>>(P);
  count_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  tpp_ctx v = *c;                 // the second stage: the 2D steps on the first E factor sets
  v.E = c->sys_E;
  return launch_factor_inverse(&v, s);
}

cudaError_t launch_full3_apply(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                               cudaStream_t s) {
  const int n = c->n, m = 5 * n;
  const size_t smem = (size_t)(m * m + m * n * n) * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(k_full3_apply_z,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_full3_apply_z<<<(unsigned)c->sys_E, 256, smem, s>>>(n, c->p<double>(c->fb.inv), b, x, skip);
  count_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  tpp_ctx v = *c;                 // the y-x factor on each of the 5n slices of an element
  v.dim = 3;
  v.R = 5;
  v.EB = c->sys_E * 5;
  return launch_apply_2d(&v, x, x, TPP_FP64, skip, s);
}

cudaError_t launch_full_build(const tpp_ctx* c, cudaStream_t s) {
  const int n = c->n, m = kNcFull * n;
  const int64_t E = c->sys_E;
  DevStatus* st = c->p<DevStatus>(c->L.status);
  FullArgs a;
  a.T = c->p<Tables>(c->L.tables);
  a.n = n;
  a.E = E;
  a.hd = c->prob.h * c->prob.h;
  a.cx = c->p<double>(c->sys_cx);
  a.cy = c->p<double>(c->sys_cy);
  a.fo = c->p<double>(c->sys_fo);
  a.QB = c->p<double>(c->fb.QB);
  a.RB = c->p<double>(c->fb.RB);
  a.rk = c->p<int32_t>(c->fb.rk);
  a.A = c->p<double>(c->fb.A);
  a.B = c->p<double>(c->fb.B);
  a.sig = c->p<double>(c->fb.sig);
  a.flags = c->p<int32_t>(c->fb.flags);
  a.st = st;
  size_t smem = (size_t)full_ksvd_smem(n).total * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(k_full_ksvd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  k_full_ksvd<<<(unsigned)E, 256, smem, s>>>(a);
  count_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const int ld = ld_of(n);
  smem = (size_t)4 * (2 * n * n + 2 * n * ld + 2 * n + 8) * sizeof(double);
  err = cudaFuncSetAttribute(k_full_bside, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_full_bside<<<(unsigned)((E + 3) / 4), 128, smem, s>>>(
      n, E, a.B, c->p<double>(c->fb.T), c->p<double>(c->fb.Q), c->p<double>(c->fb.Mb), a.flags,
      st);
  count_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const int dm = 2 * m;
  smem = (size_t)(dm * dm + dm + 16 + (dm + 1) / 2 + 1) * sizeof(double);
  err = cudaFuncSetAttribute(k_full_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_full_shift<<<(unsigned)(E * n), 256, smem, s>>>(n, E, a.A, c->p<double>(c->fb.T),
                                                      c->p<double>(c->fb.inv), a.flags, st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_full_apply(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                              cudaStream_t s) {
  const int n = c->n, m = kNcFull * n;
  FullApplyArgs P;
  P.n = n;
  P.E = c->sys_E;
  P.T = c->p<double>(c->fb.T);
  P.Q = c->p<double>(c->fb.Q);
  P.Mb = c->p<double>(c->fb.Mb);
  P.A = c->p<double>(c->fb.A);
  P.inv = c->p<double>(c->fb.inv);
  P.b = b;
  P.x = x;
  P.skip = skip;
  const size_t smem = (size_t)(4 * m * n + m * m + 3 * n * n + 2 * m) * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(k_full_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  k_full_apply<<<(unsigned)c->sys_E, 256, smem, s>>>(P);
  count_launch();
  return cudaGetLastError();
}

// rows of a full block: n_c n^dim
static int full_nb(const tpp_ctx* c) {
  return c->sys_nc * (c->dim == 2 ? c->n * c->n : c->n * c->n * c->n);
}

cudaError_t launch_full_bj_build(const tpp_ctx* c, cudaStream_t s) {
  const int n = c->n;
  const double h = c->prob.h;
  if (c->dim == 2)
    k_full_bj_assemble<<<(unsigned)c->sys_E, 256, 0, s>>>(
        c->p<Tables>(c->L.tables), n, h * h, c->p<double>(c->sys_cx), c->p<double>(c->sys_cy),
        c->p<double>(c->sys_fo), c->p<double>(c->fb.lu));
  else
    k_full_bj_assemble_3d<<<(unsigned)c->sys_E, 256, 0, s>>>(
        c->p<Tables>(c->L.tables), n, h * h * h, c->p<double>(c->sys_cx),
        c->p<double>(c->sys_cy), c->p<double>(c->sys_cz), c->p<double>(c->sys_fo),
        c->p<double>(c->fb.lu));
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_bj_lu(full_nb(c), c->sys_E, c->p<double>(c->fb.lu), c->p<int32_t>(c->fb.piv), s);
}

cudaError_t launch_full_bj_apply(const tpp_ctx* c, const double* b, double* x,
                                 const int32_t* skip, cudaStream_t s) {
  return launch_bj_solve(full_nb(c), c->sys_E, 1, c->p<double>(c->fb.lu),
                         c->p<int32_t>(c->fb.piv), b, x, skip, s);
}

}  // namespace tpp
