// Small per-problem kernels (one thread block per problem of a batch).
//
//  k_chol     FP32 Cholesky of the Gram X^* X with diagonal pivoting: the R factor of a
//             column-pivoted QR (Algorithm 3, lines with QR / QR with column pivoting),
//             the rank criterion ||R(i:r0,i:r0)||_F <= tol ||R||_F (Section 2.2) read off the
//             trailing Schur-complement trace, and the map X -> X P R^{-1}.
//  k_svd_S    FP64 one-sided Jacobi SVD of Q = U^* T V (Algorithm 3, final step) and
//             S_l = U_Q^* (U^* T_l V) V_Q Sigma^{-1} (Eq. generateSl).
//  k_eig_t    FP64: C_mu = sum_l mu_l S_l, Hessenberg reduction + shifted complex QR +
//             triangular eigenvectors -> W; z_j(l) = (W^{-1} S_l W)_jj (Eq. diagonalizeSl);
//             t_j(l) = -arg z_j(l) / 2 pi mod 1 (Algorithm 1, principal logarithm).
//  k_solve_c  FP64 Vandermonde Gram conj(A) A^T (product of Dirichlet kernels) and Cholesky
//             solve of the normal equations of Eq. ls_probl; results sorted by t.
// All loops are bounded; a cap that is hit sets PRONY_ENOCONV in the problem's state.
#include "common.cuh"
#include <algorithm>

#define ST_OK 0
#define ST_ERANK (-2)
#define ST_ENOCONV (-3)
#define ST_ENAN (-4)

namespace {

__device__ inline int swidth(const ProbState& s, const ProbDesc& p, int sel) {
  switch (sel) {
    case W_R0: return p.r0;
    case W_U: return s.wu;
    case W_V: return s.wv;
    case W_M: return p.m;
    case W_IN: return s.w_in;
    default: return s.w_out;
  }
}
__device__ inline void set_width(ProbState& s, int sel, int w) {
  if (sel == W_U) s.wu = w;
  else if (sel == W_V) s.wv = w;
}
__device__ inline void set_status(ProbState& s, int st) {
  if (s.status == ST_OK) s.status = st;
}

// ----------------------------------------------------------------------------- pivoted Cholesky (FP32)
__global__ void __launch_bounds__(256) k_chol(Dev D, int wsel, int target, int mode, double tol, int rank_mode) {
  extern __shared__ float2 A[];                 // [w][LDR]
  __shared__ int perm[PRONY_RMAX];
  __shared__ float red_v[256];
  __shared__ int red_i[256];
  __shared__ int s_piv, s_stop, s_rho, s_rank;
  __shared__ float s_trace0, s_maxd0;
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (st.done) return;
  const int w = swidth(st, p, wsel);
  const int LR = D.L.LDR;
  const double2* G = (const double2*)(D.small + p.soff + D.L.gram);
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    int i = idx / w, j = idx % w;
    double2 g = G[i * LR + j];
    A[i * LR + j] = make_float2((float)g.x, (float)g.y);
  }
  for (int i = threadIdx.x; i < w; i += blockDim.x) perm[i] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tr = 0.f, mx = 0.f;
    for (int i = 0; i < w; ++i) {
      float dd = A[i * LR + i].x;
      tr += fmaxf(dd, 0.f);
      mx = fmaxf(mx, dd);
    }
    s_trace0 = tr;
    s_maxd0 = mx;
    s_rho = w;
    s_rank = -1;
    s_stop = 0;
  }
  __syncthreads();
  const float tol2 = (float)(tol * tol);
  int limit = w;  // columns that may be accepted (never more than m after the rank step)
  if (mode == QR_RANK) limit = min(w, p.m);
  for (int i = 0; i < w; ++i) {
    // pivot search and trailing trace
    float best = -1.f;
    int bi = i;
    float tr = 0.f;
    for (int j = i + threadIdx.x; j < w; j += blockDim.x) {
      float dd = A[j * LR + j].x;
      tr += fmaxf(dd, 0.f);
      if (dd > best) { best = dd; bi = j; }
    }
    red_v[threadIdx.x] = best;
    red_i[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        float v2 = red_v[threadIdx.x + o];
        int i2 = red_i[threadIdx.x + o];
        if (v2 > red_v[threadIdx.x] || (v2 == red_v[threadIdx.x] && i2 < red_i[threadIdx.x])) {
          red_v[threadIdx.x] = v2;
          red_i[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    // trailing trace
    float trs = tr;
    for (int o = 16; o > 0; o >>= 1) trs += __shfl_xor_sync(0xffffffffu, trs, o);
    __shared__ float tr_w[8];
    if ((threadIdx.x & 31) == 0) tr_w[threadIdx.x >> 5] = trs;
    __syncthreads();
    if (threadIdx.x == 0) {
      float trail = 0.f;
      for (int q = 0; q < 8; ++q) trail += tr_w[q];
      int pv = (mode == QR_PLAIN) ? i : red_i[0];
      float dp = A[pv * LR + pv].x;
      if (mode == QR_RANK && s_rank < 0 && trail <= tol2 * s_trace0) s_rank = i;
      bool stop = false;
      if (!(dp > 1e-30f * s_maxd0) || !(dp > 0.f)) stop = true;                    // exhausted / not PD
      if (mode == QR_DROP && dp <= tol2 * s_maxd0) stop = true;
      if (i >= limit && (mode != QR_RANK || s_rank >= 0)) stop = true;
      if (mode == QR_RANK && rank_mode == 1 && s_rank >= 0) stop = true;
      if (stop) {
        s_stop = 1;
        s_rho = min(i, limit);
      }
      s_piv = pv;
    }
    __syncthreads();
    if (s_stop) break;
    const int pv = s_piv;
    if (i >= limit) {
      // beyond the accepted columns: only continue the factorisation to locate the rank
    }
    if (pv != i) {
      for (int j = threadIdx.x; j < w; j += blockDim.x) {  // swap rows i, pv
        float2 t = A[i * LR + j];
        A[i * LR + j] = A[pv * LR + j];
        A[pv * LR + j] = t;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < w; j += blockDim.x) {  // swap cols i, pv
        float2 t = A[j * LR + i];
        A[j * LR + i] = A[j * LR + pv];
        A[j * LR + pv] = t;
      }
      if (threadIdx.x == 0) {
        int t = perm[i];
        perm[i] = perm[pv];
        perm[pv] = t;
      }
      __syncthreads();
    }
    const float lii = sqrtf(A[i * LR + i].x);
    __syncthreads();
    for (int j = i + 1 + threadIdx.x; j < w; j += blockDim.x) {
      float2 v = A[j * LR + i];
      A[j * LR + i] = make_float2(v.x / lii, v.y / lii);
    }
    if (threadIdx.x == 0) A[i * LR + i] = make_float2(lii, 0.f);
    __syncthreads();
    const int rem = w - i - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      int j = i + 1 + idx / rem, k = i + 1 + idx % rem;
      float2 lj = A[j * LR + i], lk = A[k * LR + i];
      float2 a = A[j * LR + k];
      a.x -= lj.x * lk.x + lj.y * lk.y;            // lj * conj(lk)
      a.y -= lj.y * lk.x - lj.x * lk.y;
      A[j * LR + k] = a;
    }
    __syncthreads();
  }
  __syncthreads();
  const int rho = min(s_rho, limit);
  // R = L^H (rho x rho); M[perm[a]][b] = Rinv[a][b]; Rinv by column back substitution.
  float2* M = (float2*)(D.small + p.soff + D.L.mapm);
  for (int idx = threadIdx.x; idx < w * max(rho, 1); idx += blockDim.x) {
    int i = idx / max(rho, 1), j = idx % max(rho, 1);
    M[i * LR + j] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < rho; b += blockDim.x) {
    float2 x[PRONY_RMAX];
    for (int a = b; a >= 0; --a) {
      float2 s = (a == b) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
      for (int k = a + 1; k <= b; ++k) {
        float2 l = A[k * LR + a];            // R[a][k] = conj(L[k][a])
        float2 xk = x[k];
        s.x -= l.x * xk.x + l.y * xk.y;
        s.y -= l.x * xk.y - l.y * xk.x;
      }
      float r = A[a * LR + a].x;
      x[a] = make_float2(s.x / r, s.y / r);
    }
    for (int a = 0; a <= b; ++a) M[perm[a] * LR + b] = x[a];
  }
  if (threadIdx.x == 0) {
    st.w_in = w;
    st.w_out = rho;
    set_width(st, target, rho);
    if (mode == QR_RANK) {
      st.rank_det = s_rank >= 0 ? s_rank : w;
      st.rank_used = rho;
      if (rho < p.m) set_status(st, ST_ERANK);
    }
    if (rho == 0) {
      set_status(st, ST_ERANK);
      st.done = 1;
    }
  }
}

// ----------------------------------------------------------------------------- Jacobi SVD + S_l (FP64)
__device__ inline void rr_pair(int step, int k, int nb, int& pa, int& pb) {
  // circle method: position 0 fixed, positions 1..nb-1 rotate
  auto who = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + step) % (nb - 1)) + 1; };
  pa = who(k);
  pb = who(nb - 1 - k);
}

__global__ void __launch_bounds__(256) k_svd_S(Dev D) {
  extern __shared__ double2 sm[];
  __shared__ int s_rot;
  __shared__ double s_sig[PRONY_MMAX];
  __shared__ int s_rank[PRONY_MMAX];
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (st.status == ST_ENAN) return;
  const int a = st.wu, b = st.wv;
  if (b <= 0) return;
  double2* Qc = sm;                                  // [b][a] columns
  double2* Vc = sm + (size_t)D.L.LDM * D.L.LDR;      // [b][b] columns
  const int LM = D.L.LDM, LR = D.L.LDR;
  const double2* Q = (const double2*)(D.small + p.soff + D.L.q);
  for (int idx = threadIdx.x; idx < a * b; idx += blockDim.x) {
    int i = idx % a, j = idx / a;
    Qc[j * a + i] = Q[i * LM + j];
  }
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    int i = idx % b, j = idx / b;
    Vc[j * b + i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const int nb = b + (b & 1);
  const double jtol = 4.0 * a * 2.220446049250313e-16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step < nb - 1; ++step) {
      for (int k = warp; k < nb / 2; k += nwarp) {
        int pa, pb;
        rr_pair(step, k, nb, pa, pb);
        if (pa >= b || pb >= b) continue;
        if (pa > pb) { int t = pa; pa = pb; pb = t; }
        double al = 0.0, be = 0.0;
        double2 ga = make_double2(0.0, 0.0);
        for (int i = lane; i < a; i += 32) {
          double2 x = Qc[pa * a + i], y = Qc[pb * a + i];
          al += cabs2(x);
          be += cabs2(y);
          ga = cadd(ga, cmulc(x, y));
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
        }
        double ag = sqrt(cabs2(ga));
        if (ag <= jtol * sqrt(al * be) || ag == 0.0) continue;
        double zeta = (be - al) / (2.0 * ag);
        double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
        double2 ph = make_double2(ga.x / ag, -ga.y / ag);   // e^{-i phi}
        for (int i = lane; i < a; i += 32) {
          double2 x = Qc[pa * a + i], y = cmul(Qc[pb * a + i], ph);
          Qc[pa * a + i] = csub(cscale(x, c), cscale(y, s));
          Qc[pb * a + i] = cadd(cscale(x, s), cscale(y, c));
        }
        for (int i = lane; i < b; i += 32) {
          double2 x = Vc[pa * b + i], y = cmul(Vc[pb * b + i], ph);
          Vc[pa * b + i] = csub(cscale(x, c), cscale(y, s));
          Vc[pb * b + i] = cadd(cscale(x, s), cscale(y, c));
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  // singular values (column norms), descending order
  for (int j = warp; j < b; j += nwarp) {
    double s2 = 0.0;
    for (int i = lane; i < a; i += 32) s2 += cabs2(Qc[j * a + i]);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) s_sig[j] = sqrt(s2);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < b; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < b; ++i)
      if (s_sig[i] > s_sig[j] || (s_sig[i] == s_sig[j] && i < j)) ++r;
    s_rank[j] = r;
  }
  __syncthreads();
  double2* UQ = (double2*)(D.small + p.soff + D.L.uq);
  double2* VQ = (double2*)(D.small + p.soff + D.L.vq);
  double* sig = (double*)(D.small + p.soff + D.L.sigma);
  for (int idx = threadIdx.x; idx < a * b; idx += blockDim.x) {
    int i = idx % a, j = idx / a;
    double sj = s_sig[j];
    double2 v = Qc[j * a + i];
    UQ[i * LM + s_rank[j]] = sj > 0.0 ? cscale(v, 1.0 / sj) : make_double2(0.0, 0.0);
  }
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    int i = idx % b, j = idx / b;
    VQ[i * LM + s_rank[j]] = Vc[j * b + i];
  }
  for (int j = threadIdx.x; j < b; j += blockDim.x) sig[s_rank[j]] = s_sig[j];
  if (threadIdx.x == 0 && sweep >= 40) set_status(st, ST_ENOCONV);
  __syncthreads();
  // S_l = UQ^H (M_l VQ) Sigma^{-1}
  double2* tmp = sm;  // reuse: [a][b]
  for (int l = 0; l < p.d; ++l) {
    const double2* Ml = (const double2*)(D.small + p.soff + D.L.mproj) + (size_t)l * LR * LM;
    __syncthreads();
    for (int idx = threadIdx.x; idx < a * b; idx += blockDim.x) {
      int i = idx / b, j = idx % b;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < b; ++k) acc = cadd(acc, cmul(Ml[i * LM + k], VQ[k * LM + j]));
      tmp[i * b + j] = acc;
    }
    __syncthreads();
    double2* S = (double2*)(D.small + p.soff + D.L.S) + (size_t)l * LM * LM;
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
      int i = idx / b, j = idx % b;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < a; ++k) acc = cadd(acc, cmulc(UQ[k * LM + i], tmp[k * b + j]));
      double sj = sig[j];
      S[i * LM + j] = sj > 0.0 ? cscale(acc, 1.0 / sj) : make_double2(0.0, 0.0);
    }
  }
  if (threadIdx.x == 0) {
    double s0 = s_sig[0];
    for (int j = 1; j < b; ++j) s0 = fmax(s0, s_sig[j]);
    double smin = s0;
    for (int j = 0; j < b; ++j) smin = fmin(smin, s_sig[j]);
    st.sigma_ratio = s0 > 0.0 ? smin / s0 : 0.0;
  }
}

// Canonical phases: ph_j = v_j[argmax] / |.|;  S_l <- D^* S_l D with D = diag(conj ph);
// U_Q, V_Q columns times conj(ph).  V_final = V V_Q is in buffer `buf` (argmax done).
__global__ void k_canon(Dev D) {
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  const int b = st.wv, a = st.wu;
  __shared__ double2 ph[PRONY_MMAX];
  const int LM = D.L.LDM;
  const unsigned long long* am = (const unsigned long long*)(D.small + p.soff + D.L.argmx);
  for (int j = threadIdx.x; j < b; j += blockDim.x) {
    unsigned row = am[j] == 0ull ? 0u : 0xFFFFFFFFu - (unsigned)(am[j] & 0xFFFFFFFFull);
    if (row >= (unsigned)p.N) row = 0u;
    float2 v = D.B1[p.xoff + (long long)j * p.N + row];
    double r = hypot((double)v.x, (double)v.y);
    ph[j] = r > 0.0 ? make_double2(v.x / r, v.y / r) : make_double2(1.0, 0.0);
    ((double2*)(D.small + p.soff + D.L.phase))[j] = ph[j];
  }
  __syncthreads();
  for (int l = 0; l < p.d; ++l) {
    double2* S = (double2*)(D.small + p.soff + D.L.S) + (size_t)l * LM * LM;
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
      int i = idx / b, j = idx % b;
      S[i * LM + j] = cmul(cmul(ph[i], S[i * LM + j]), cconj(ph[j]));
    }
  }
  double2* UQ = (double2*)(D.small + p.soff + D.L.uq);
  double2* VQ = (double2*)(D.small + p.soff + D.L.vq);
  for (int idx = threadIdx.x; idx < a * b; idx += blockDim.x) {
    int i = idx / b, j = idx % b;
    UQ[i * LM + j] = cmul(UQ[i * LM + j], cconj(ph[j]));
  }
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    int i = idx / b, j = idx % b;
    VQ[i * LM + j] = cmul(VQ[i * LM + j], cconj(ph[j]));
  }
}

// ----------------------------------------------------------------------------- eigen step (FP64)
__device__ inline double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

__global__ void __launch_bounds__(256) k_eig_t(Dev D, unsigned long long seed) {
  extern __shared__ double2 sm[];
  __shared__ double2 mu[PRONY_DMAX];
  __shared__ double2 hv[PRONY_MMAX];
  __shared__ double2 sv[PRONY_MMAX];
  __shared__ double s_norm;
  __shared__ int s_fail;
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (st.status == ST_ENAN) return;
  const int m = st.wv;
  if (m <= 0) return;
  const int LD = D.L.LDM;
  double2* H = sm;                     // [m][LD]
  double2* Z = sm + LD * LD;           // [m][LD]
  double2* Y = Z + LD * LD;            // eigenvectors of the triangular factor, later W^{-1}
  const double2* S = (const double2*)(D.small + p.soff + D.L.S);
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int l = 0; l < p.d; ++l) {
      uint64_t c[4] = {(uint64_t)l, 0, 0, 0};
      philox4x64(c, seed, PRONY_STREAM_MU);
      double u0 = philox_u01(c[0]), u1 = philox_u01(c[1]);
      double r = sqrt(-log(u0)), sn, cs;
      sincospi(2.0 * u1, &sn, &cs);
      mu[l] = make_double2(r * cs, r * sn);
      nrm += cabs2(mu[l]);
    }
    nrm = sqrt(nrm);
    for (int l = 0; l < p.d; ++l) mu[l] = cscale(mu[l], 1.0 / nrm);
    s_fail = 0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < p.d; ++l) acc = cadd(acc, cmul(mu[l], S[(size_t)l * LD * LD + i * LD + j]));
    H[i * LD + j] = acc;
    Z[i * LD + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // --- Householder reduction to upper Hessenberg form, H <- Q^H H Q, Z <- Z Q
  for (int k = 0; k + 2 < m; ++k) {
    if (threadIdx.x == 0) {
      double nx = 0.0;
      for (int i = k + 1; i < m; ++i) nx += cabs2(H[i * LD + k]);
      nx = sqrt(nx);
      double2 x0 = H[(k + 1) * LD + k];
      double ax0 = sqrt(cabs2(x0));
      double2 ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
      double2 alpha = cscale(ph, -nx);                 // alpha = -e^{i arg x0} ||x||
      for (int i = 0; i < m; ++i) hv[i] = make_double2(0.0, 0.0);
      for (int i = k + 1; i < m; ++i) hv[i] = H[i * LD + k];
      hv[k + 1] = csub(hv[k + 1], alpha);
      double nv = 0.0;
      for (int i = k + 1; i < m; ++i) nv += cabs2(hv[i]);
      s_norm = nv;
      if (nv > 0.0) {
        double inv = 1.0 / sqrt(nv);
        for (int i = k + 1; i < m; ++i) hv[i] = cscale(hv[i], inv);
      }
    }
    __syncthreads();
    if (s_norm > 0.0) {
      // left: H[k+1:, j] -= 2 v (v^H H[k+1:, j])
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int i = k + 1; i < m; ++i) s = cadd(s, cmulc(hv[i], H[i * LD + j]));
        sv[j] = s;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < (m - k - 1) * m; idx += blockDim.x) {
        int i = k + 1 + idx / m, j = idx % m;
        H[i * LD + j] = csub(H[i * LD + j], cscale(cmul(hv[i], sv[j]), 2.0));
      }
      __syncthreads();
      // right: H[i, k+1:] -= 2 (H[i, k+1:] v) v^H ; Z likewise
      for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
        double2* R = i < m ? H : Z;
        int ii = i < m ? i : i - m;
        double2 s = make_double2(0.0, 0.0);
        for (int j = k + 1; j < m; ++j) s = cadd(s, cmul(R[ii * LD + j], hv[j]));
        for (int j = k + 1; j < m; ++j) R[ii * LD + j] = csub(R[ii * LD + j], cscale(cmul(s, cconj(hv[j])), 2.0));
      }
      __syncthreads();
      for (int i = k + 2 + threadIdx.x; i < m; i += blockDim.x) H[i * LD + k] = make_double2(0.0, 0.0);
      __syncthreads();
    }
  }
  // --- shifted complex QR iteration on the Hessenberg matrix (one warp), full Schur form
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double eps = 2.220446049250313e-16;
    int hi = m - 1, its = 0, total = 0;
    const int cap = 30 * m + 30;
    while (hi > 0) {
      if (total > cap) break;
      int l = hi;
      for (; l > 0; --l) {
        double s = cabs1(H[(l - 1) * LD + l - 1]) + cabs1(H[l * LD + l]);
        if (s == 0.0) s = 1.0;
        if (cabs1(H[l * LD + l - 1]) <= eps * s) break;
      }
      if (l > 0 && lane == 0) H[l * LD + l - 1] = make_double2(0.0, 0.0);
      __syncwarp();
      if (l == hi) {
        --hi;
        its = 0;
        continue;
      }
      // shift
      double2 sh;
      if (its == 10 || its == 20) {
        sh = cadd(H[hi * LD + hi], make_double2(0.75 * cabs1(H[hi * LD + hi - 1]), 0.0));
      } else {
        double2 a = H[(hi - 1) * LD + hi - 1], bb = H[(hi - 1) * LD + hi], c = H[hi * LD + hi - 1], d = H[hi * LD + hi];
        double2 hd = cscale(csub(a, d), 0.5);
        double2 disc = csqrtd(cadd(cmul(hd, hd), cmul(bb, c)));
        double2 mid = cscale(cadd(a, d), 0.5);
        double2 l1 = cadd(mid, disc), l2 = csub(mid, disc);
        sh = cabs2(csub(l1, d)) <= cabs2(csub(l2, d)) ? l1 : l2;
      }
      // implicit single-shift QR sweep on rows/cols l..hi
      double2 x = csub(H[l * LD + l], sh), y = H[(l + 1) * LD + l];
      for (int k = l; k < hi; ++k) {
        if (k > l) {
          x = H[k * LD + k - 1];
          y = H[(k + 1) * LD + k - 1];
        }
        double ax = sqrt(cabs2(x)), ay = sqrt(cabs2(y));
        double nr = hypot(ax, ay);
        double c;
        double2 s;
        if (nr == 0.0) {
          c = 1.0;
          s = make_double2(0.0, 0.0);
        } else if (ax == 0.0) {
          c = 0.0;
          s = cscale(cconj(y), 1.0 / ay);
        } else {
          c = ax / nr;
          s = cscale(cmul(cscale(x, 1.0 / ax), cconj(y)), 1.0 / nr);
        }
        // rows k, k+1 : [r_k; r_k1] <- [c s; -conj(s) c] [r_k; r_k1], columns from max(l, k-1)
        for (int j = max(l, k - 1) + lane; j < m; j += 32) {
          double2 rk = H[k * LD + j], rk1 = H[(k + 1) * LD + j];
          H[k * LD + j] = cadd(cscale(rk, c), cmul(s, rk1));
          H[(k + 1) * LD + j] = csub(cscale(rk1, c), cmul(cconj(s), rk));
        }
        __syncwarp();
        // columns k, k+1 : H <- H G^H, rows 0 .. min(k+2, hi)
        int rmax = min(k + 2, hi);
        for (int i = lane; i <= rmax; i += 32) {
          double2 ck = H[i * LD + k], ck1 = H[i * LD + k + 1];
          H[i * LD + k] = cadd(cscale(ck, c), cmul(cconj(s), ck1));
          H[i * LD + k + 1] = csub(cscale(ck1, c), cmul(s, ck));
        }
        for (int i = lane; i < m; i += 32) {
          double2 ck = Z[i * LD + k], ck1 = Z[i * LD + k + 1];
          Z[i * LD + k] = cadd(cscale(ck, c), cmul(cconj(s), ck1));
          Z[i * LD + k + 1] = csub(cscale(ck1, c), cmul(s, ck));
        }
        __syncwarp();
      }
      ++its;
      ++total;
    }
    if (lane == 0 && hi > 0) s_fail = 1;
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0) set_status(st, ST_ENOCONV);
  // --- eigenvectors of the triangular Schur factor: (T - lambda_k I) y = 0, y_k = 1
  double hn = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i)
      for (int j = i; j < m; ++j) hn = fmax(hn, cabs1(H[i * LD + j]));
    s_norm = hn;
  }
  __syncthreads();
  const double small = fmax(s_norm, 1e-300) * 2.220446049250313e-16;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    double2 lam = H[k * LD + k];
    for (int i = k + 1; i < m; ++i) Y[i * LD + k] = make_double2(0.0, 0.0);
    Y[k * LD + k] = make_double2(1.0, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double2 s = make_double2(0.0, 0.0);
      for (int j = i + 1; j <= k; ++j) s = cadd(s, cmul(H[i * LD + j], Y[j * LD + k]));
      double2 den = csub(H[i * LD + i], lam);
      if (cabs1(den) < small) den = make_double2(small, 0.0);
      Y[i * LD + k] = cdiv(make_double2(-s.x, -s.y), den);
    }
  }
  __syncthreads();
  // W = Z Y (columns normalised); store W in H's storage
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, k = idx % m;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j <= k; ++j) acc = cadd(acc, cmul(Z[i * LD + j], Y[j * LD + k]));
    H[i * LD + k] = acc;  // H no longer needed
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += cabs2(H[i * LD + k]);
    sv[k] = make_double2(s > 0.0 ? 1.0 / sqrt(s) : 1.0, 0.0);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, k = idx % m;
    H[i * LD + k] = cscale(H[i * LD + k], sv[k].x);
  }
  __syncthreads();
  // --- W^{-1} by Gauss-Jordan with partial pivoting: Z <- W (copy), Y <- I
  double2* Wm = H;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    Z[i * LD + j] = Wm[i * LD + j];
    Y[i * LD + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __shared__ int s_pr;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      int pr = k;
      double best = cabs1(Z[k * LD + k]);
      for (int i = k + 1; i < m; ++i) {
        double v = cabs1(Z[i * LD + k]);
        if (v > best) { best = v; pr = i; }
      }
      s_pr = pr;
      if (best == 0.0) s_fail = 2;
    }
    __syncthreads();
    const int pr = s_pr;
    if (pr != k) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double2 t = Z[k * LD + j]; Z[k * LD + j] = Z[pr * LD + j]; Z[pr * LD + j] = t;
        t = Y[k * LD + j]; Y[k * LD + j] = Y[pr * LD + j]; Y[pr * LD + j] = t;
      }
      __syncthreads();
    }
    double2 piv = Z[k * LD + k];
    if (cabs1(piv) == 0.0) piv = make_double2(1e-300, 0.0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      Z[k * LD + j] = cdiv(Z[k * LD + j], piv);
      Y[k * LD + j] = cdiv(Y[k * LD + j], piv);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) hv[i] = (i == k) ? make_double2(0.0, 0.0) : Z[i * LD + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = idx / m, j = idx % m;
      if (i == k) continue;
      double2 f = hv[i];
      Z[i * LD + j] = csub(Z[i * LD + j], cmul(f, Z[k * LD + j]));
      Y[i * LD + j] = csub(Y[i * LD + j], cmul(f, Y[k * LD + j]));
    }
    __syncthreads();
  }
  __syncthreads();
  // Y = W^{-1};  z_j(l) = sum_a Winv[j][a] (S_l W)[a][j];  t = -arg z / 2pi mod 1
  double* tout = (double*)(D.small + p.soff + D.L.t);
  for (int l = 0; l < p.d; ++l) {
    const double2* Sl = S + (size_t)l * LD * LD;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {   // Z <- S_l W
      int i = idx / m, j = idx % m;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < m; ++k) acc = cadd(acc, cmul(Sl[i * LD + k], Wm[k * LD + j]));
      Z[i * LD + j] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      double2 z = make_double2(0.0, 0.0);
      for (int a = 0; a < m; ++a) z = cadd(z, cmul(Y[j * LD + a], Z[a * LD + j]));
      double tj = -atan2(z.y, z.x) / 6.283185307179586;
      tj -= floor(tj);
      if (tj >= 1.0) tj = 0.0;
      tout[j * PRONY_DMAX + l] = tj;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_fail == 2) set_status(st, ST_ENOCONV);
  if (threadIdx.x == 0) st.rank_used = m;
}

// ----------------------------------------------------------------------------- c by normal equations (FP64)
__global__ void __launch_bounds__(256) k_solve_c(Dev D) {
  extern __shared__ double2 G[];                     // [m][MMAX]
  __shared__ double2 bb[PRONY_MMAX];
  __shared__ double ts[PRONY_MMAX * PRONY_DMAX];
  __shared__ int s_bad;
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  const int m = st.rank_used, d = p.d, LD = PRONY_MMAX;
  if (m <= 0) return;
  double* t = (double*)(D.small + p.soff + D.L.t);
  double2* b = (double2*)(D.small + p.soff + D.L.rhs);
  double2* cout = (double2*)(D.small + p.soff + D.L.c);
  for (int q = threadIdx.x; q < m * d; q += blockDim.x) ts[(q / d) * PRONY_DMAX + q % d] = t[(q / d) * PRONY_DMAX + q % d];
  for (int i = threadIdx.x; i < m; i += blockDim.x) bb[i] = b[i];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // G[i][j] = prod_l sum_{x=0}^{n} exp(2 pi i (t_i(l) - t_j(l)) x)
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    double2 g = make_double2(1.0, 0.0);
    for (int l = 0; l < d; ++l) {
      double dl = ts[i * PRONY_DMAX + l] - ts[j * PRONY_DMAX + l];
      dl -= rint(dl);
      double2 term;
      if (dl == 0.0) {
        term = make_double2((double)(p.n + 1), 0.0);
      } else {
        double num = sinpi(dl * (p.n + 1)), den = sinpi(dl), sn, cs;
        sincospi(dl * p.n, &sn, &cs);
        term = cscale(make_double2(cs, sn), num / den);
      }
      g = cmul(g, term);
    }
    G[i * LD + j] = g;
  }
  __syncthreads();
  // Cholesky G = L L^H (lower, in place), single thread per row update
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double dkk = G[k * LD + k].x;
      if (!(dkk > 0.0)) { s_bad = 1; dkk = 1e-300; }
      G[k * LD + k] = make_double2(sqrt(dkk), 0.0);
    }
    __syncthreads();
    double lkk = G[k * LD + k].x;
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) G[i * LD + k] = cscale(G[i * LD + k], 1.0 / lkk);
    __syncthreads();
    int rem = m - k - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j > i) continue;
      G[i * LD + j] = csub(G[i * LD + j], cmul(G[i * LD + k], cconj(G[j * LD + k])));
    }
    __syncthreads();
  }
  __shared__ double2 cs_[PRONY_MMAX];
  if (threadIdx.x == 0) {
    // L y = b ; L^H c = y
    for (int i = 0; i < m; ++i) {
      double2 s = bb[i];
      for (int k = 0; k < i; ++k) s = csub(s, cmul(G[i * LD + k], cs_[k]));
      cs_[i] = cscale(s, 1.0 / G[i * LD + i].x);
    }
    for (int i = m - 1; i >= 0; --i) {
      double2 s = cs_[i];
      for (int k = i + 1; k < m; ++k) s = csub(s, cmul(cconj(G[k * LD + i]), cs_[k]));
      cs_[i] = cscale(s, 1.0 / G[i * LD + i].x);
    }
    if (s_bad) set_status(st, ST_ERANK);
  }
  __syncthreads();
  // sort (t, c) lexicographically by t
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < m; ++i) {
      bool less = false, eq = true;
      for (int l = 0; l < d && eq; ++l) {
        double a = ts[i * PRONY_DMAX + l], bq = ts[j * PRONY_DMAX + l];
        if (a < bq) { less = true; eq = false; }
        else if (a > bq) { eq = false; }
      }
      if (less || (eq && i < j)) ++r;
    }
    for (int l = 0; l < d; ++l) t[r * PRONY_DMAX + l] = ts[j * PRONY_DMAX + l];
    cout[r] = cs_[j];
  }
  if (threadIdx.x == 0) st.ls_num2 = 0.0;
}

// ----------------------------------------------------------------------------- convergence check
__global__ void k_check(Dev D, double tol_power, int max_iter, int* all_done) {
  int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= D.nprob) return;
  ProbState& s = D.st[pi];
  if (s.nonfinite) {
    s.status = ST_ENAN;
    s.done = 1;
  }
  if (s.done) return;
  s.iter += 1;
  double r2 = s.resid2, t2 = tol_power * tol_power * s.normT2;
  bool conv = r2 <= t2;
  bool stagn = s.resid2_prev >= 0.0 && r2 >= 0.64 * s.resid2_prev;
  bool nan = !(r2 == r2);
  if (nan) {
    s.status = ST_ENAN;
    s.done = 1;
  } else if (conv || stagn) {
    s.done = 1;
  } else if (s.iter >= max_iter) {
    set_status(s, ST_ENOCONV);
    s.done = 1;
  } else {
    s.resid2_prev = r2;
    s.resid2 = 0.0;
  }
  if (!s.done) atomicExch(all_done, 0);
}

// After the power loop: problems that stopped iterating take part in the finishing steps
// again (non-finite input stays excluded).
__global__ void k_reset_done(Dev D) {
  int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= D.nprob) return;
  ProbState& s = D.st[pi];
  s.done = (s.status == ST_ENAN || s.wv <= 0 || s.wu <= 0) ? 1 : 0;
}

}  // namespace

void launch_reset_done(const Dev& D, cudaStream_t s) { note_launch(); k_reset_done<<<(D.nprob + 127) / 128, 128, 0, s>>>(D); }

void launch_chol(const Dev& D, int wsel, int target, int mode, double tol, int rank_mode, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float2) * PRONY_RMAX * PRONY_RMAX));
    attr = true;
  }
  size_t sm = sizeof(float2) * D.L.LDR * D.L.LDR;
  note_launch();
  k_chol<<<D.nprob, 256, sm, s>>>(D, wsel, target, mode, tol, rank_mode);
}

void launch_svd_S(const Dev& D, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_svd_S, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(double2) * (PRONY_MMAX * PRONY_RMAX + PRONY_MMAX * PRONY_MMAX)));
    attr = true;
  }
  size_t sm = sizeof(double2) * ((size_t)D.L.LDM * D.L.LDR + (size_t)D.L.LDM * D.L.LDM);
  note_launch();
  k_svd_S<<<D.nprob, 256, sm, s>>>(D);
}

void launch_canon(const Dev& D, cudaStream_t s) { note_launch(); k_canon<<<D.nprob, 256, 0, s>>>(D); }

void launch_eig_t(const Dev& D, unsigned long long seed, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_eig_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double2) * 3 * PRONY_MMAX * PRONY_MMAX));
    attr = true;
  }
  size_t sm = sizeof(double2) * 3 * D.L.LDM * D.L.LDM;
  note_launch();
  k_eig_t<<<D.nprob, 256, sm, s>>>(D, seed);
}

void launch_solve_c(const Dev& D, cudaStream_t s) {
  static bool attr = false;
  size_t sm = sizeof(double2) * PRONY_MMAX * PRONY_MMAX;
  if (!attr) {
    cudaFuncSetAttribute(k_solve_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  note_launch();
  k_solve_c<<<D.nprob, 256, sm, s>>>(D);
}

void launch_check(const Dev& D, double tol_power, int max_iter, int* all_done, cudaStream_t s) {
  note_launch();
  k_check<<<(D.nprob + 127) / 128, 128, 0, s>>>(D, tol_power, max_iter, all_done);
}
