// FP64-accurate small steps of Algorithm 1, designed for GB300's FP64 unit (high latency per
// dependent operation, low throughput per SM): iterations run in FP32 on one CTA per problem,
// and the quantities that fix the results are then computed or refined in FP64 with matrix
// products only, which k_zgemm spreads over many CTAs per problem (every SM's FP64 units take
// part even when the batch has fewer problems than SMs).
//
//  SVD of Q = U^* T V (Algorithm 3, final step): k_svd_jacobi (FP32 one-sided Jacobi) gives a
//           starting V; FP64 refinement of V as eigenvectors of H = Q^*Q (Ogita & Aishima 2018,
//           iterative refinement for the symmetric eigenvalue problem based on matrix
//           multiplication, Hermitian form): per step T1 = V^*V, T2 = H V, S = V^* T2 (k_zgemm),
//           the correction F = I + E (k_oa_step), V <- V F (k_zgemm), until ||E||_F <= 1e-9;
//           k_svd_sort orders the eigenpairs, sigma = sqrt(eigenvalues); U_Q = Q V_Q Sigma^{-1}
//           and S_l = (U_Q^* (U^* T_l V)) V_Q Sigma^{-1} (Eq. generateSl) by k_zgemm.
//  Eigen step: k_eig_w forms C_mu = sum_l mu_l S_l and finds W (FP32 Hessenberg reduction,
//           shifted complex QR, triangular eigenvectors) and its FP32 inverse X; two FP64
//           Newton-Schulz steps X <- 2X - X (W X) (k_zgemm); C_l = S_l W (k_zgemm);
//           k_eig_z: z_j(l) = (X C_l)_jj, t_j(l) = -arg z_j(l) / 2pi mod 1 (Eq. diagonalizeSl).
//           The diagonal of W^{-1} S_l W is stationary in W: an error E in W (W = W_0 (I + E))
//           changes it only at second order, so z carries FP64 accuracy even though W comes
//           from FP32 iterations.
//  k_canon  phase-canonical singular basis for the S_l output.
#include "common.cuh"

#include <algorithm>


namespace {

__device__ inline void set_status_e(ProbState& s, int st) {
  if (s.status == ST_OK) s.status = st;
}

// a problem takes part in the SVD of Q: its power loop ended with a U of width a <= r0 and a V of
// width b <= m
__device__ inline bool svd_live(const ProbDesc& p, const ProbState& st) {
  return !st.done && st.status != ST_ENAN && st.wv > 0 && st.wu > 0 && st.wv <= p.m && st.wu <= p.r0;
}
// ... and in the eigen step (width m = wv of its S_l)
__device__ inline bool eig_live(const ProbDesc& p, const ProbState& st) {
  return !st.done && st.status != ST_ENAN && st.wv > 0 && st.wv <= p.m;
}

// ----------------------------------------------------------------------------- FP32 complex
__device__ inline float2 fc(float x, float y) { return make_float2(x, y); }
__device__ inline float2 fmul(float2 a, float2 b) { return fc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline float2 fmulc(float2 a, float2 b) { return fc(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ inline float2 fadd(float2 a, float2 b) { return fc(a.x + b.x, a.y + b.y); }
__device__ inline float2 fsub(float2 a, float2 b) { return fc(a.x - b.x, a.y - b.y); }
__device__ inline float2 fconj(float2 a) { return fc(a.x, -a.y); }
__device__ inline float2 fscale(float2 a, float s) { return fc(a.x * s, a.y * s); }
__device__ inline float fabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline float fabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ inline float2 fdiv(float2 a, float2 b) {
  if (fabsf(b.x) >= fabsf(b.y)) {
    float r = b.y / b.x, den = b.x + b.y * r;
    return fc((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  float r = b.x / b.y, den = b.x * r + b.y;
  return fc((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ inline float2 fsqrtc(float2 a) {
  float r = hypotf(a.x, a.y);
  if (r == 0.f) return fc(0.f, 0.f);
  float sx = sqrtf(0.5f * (r + fabsf(a.x)));
  if (a.x >= 0.f) return fc(sx, a.y / (2.f * sx));
  return fc(fabsf(a.y) / (2.f * sx), a.y >= 0.f ? sx : -sx);
}

// block-wide sum of a double (tree; result in every thread)
__device__ double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;
}

__device__ inline void rr_pair(int step, int k, int nb, int& pa, int& pb) {
  // round-robin (circle) ordering: position 0 fixed, positions 1..nb-1 rotate
  auto who = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + step) % (nb - 1)) + 1; };
  pa = who(k);
  pb = who(nb - 1 - k);
}


// ----------------------------------------------------------------------------- batched FP64 products
// C = alpha op(A) op(B) [diag(1/sigma)] [+ beta C0] for every problem of the batch (and `nl`
// consecutive matrices per problem), on the per-problem small workspace.  Matrices are row-major
// complex FP64 at byte offsets of the problem's block; op = conjugate transpose when t* = 1.
// One CTA computes a 16 x 16 tile of C: 256 threads, one entry each, K staged 16 at a time in
// shared memory; eight partial sums per entry (k mod 8) keep sixteen independent FP64 chains per
// thread in flight (a dependent FP64 operation waits hundreds of cycles on this GPU).  Dimensions come from the problem's state (a = wu, b = wv).
enum ZDim { ZD_A = 0, ZD_B = 1 };
enum ZLive { ZL_SVD = 0, ZL_EIG = 1 };
enum ZConv { ZC_ALL = 0, ZC_SKIP_CONV = 1, ZC_COPY_CONV = 2 };
struct ZG {
  long long a, b, c, c0;          // byte offsets (c0 < 0: no C0 term)
  long long la, lb, lc;           // byte strides between the nl matrices of a problem
  long long colscale;             // byte offset of sigma (< 0: no column scaling)
  int lda, ldb, ldc;
  int ta, tb;
  int M, N, K;                    // ZDim selectors
  int nl;
  int live;                       // ZLive
  int conv;                       // ZConv: skip (or copy A to C for) problems whose refinement converged
  double alpha, beta;
};
constexpr int ZT = 16;

__device__ inline int zdim(const ProbState& st, int sel) { return sel == ZD_A ? st.wu : st.wv; }

__global__ void __launch_bounds__(256) k_zgemm(Dev D, ZG g) {
  __shared__ double2 As[ZT][ZT + 1];
  __shared__ double2 Bs[ZT][ZT + 1];
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  const ProbState& st = D.st[pi];
  if (!(g.live == ZL_SVD ? svd_live(p, st) : eig_live(p, st))) return;
  const int l = blockIdx.z;
  if (l >= g.nl) return;
  const int M = zdim(st, g.M), N = zdim(st, g.N), K = zdim(st, g.K);
  const int tiles_n = (N + ZT - 1) / ZT;
  const int i0 = (blockIdx.x / tiles_n) * ZT, j0 = (blockIdx.x % tiles_n) * ZT;
  if (i0 >= M) return;
  char* sb = D.small + p.soff;
  const double2* A = (const double2*)(sb + g.a + l * g.la);
  const double2* B = (const double2*)(sb + g.b + l * g.lb);
  double2* C = (double2*)(sb + g.c + l * g.lc);
  const int ty = threadIdx.x / ZT, tx = threadIdx.x % ZT;
  const int i = i0 + ty, j = j0 + tx;
  // refinement state: 0 running, 2 last correction pending, 1 converged (products skipped, V copied)
  if ((g.conv == ZC_SKIP_CONV && st.oa_conv != 0) || (g.conv == ZC_COPY_CONV && st.oa_conv == 1)) {
    if (g.conv == ZC_COPY_CONV && i < M && j < N) C[i * g.ldc + j] = A[i * g.lda + j];
    return;
  }
  double2 acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += ZT) {
    {
      // A tile rows i0.., columns k0..; B tile rows k0.., columns j0..
      const int r = threadIdx.x / ZT, c = threadIdx.x % ZT;
      const int ai = i0 + r, ak = k0 + c;
      double2 av = make_double2(0.0, 0.0);
      if (ai < M && ak < K) av = g.ta ? cconj(A[ak * g.lda + ai]) : A[ai * g.lda + ak];
      As[r][c] = av;
      const int bk = k0 + r, bj = j0 + c;
      double2 bv = make_double2(0.0, 0.0);
      if (bk < K && bj < N) bv = g.tb ? cconj(B[bj * g.ldb + bk]) : B[bk * g.ldb + bj];
      Bs[r][c] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZT; kk += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const double2 a = As[ty][kk + u], b = Bs[kk + u][tx];
        acc[u].x = fma(a.x, b.x, acc[u].x);
        acc[u].y = fma(a.x, b.y, acc[u].y);
        acc[u].x = fma(-a.y, b.y, acc[u].x);
        acc[u].y = fma(a.y, b.x, acc[u].y);
      }
    }
    __syncthreads();
  }
  if (i >= M || j >= N) return;
  double2 v = cscale(cadd(cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3])), cadd(cadd(acc[4], acc[5]), cadd(acc[6], acc[7]))),
                     g.alpha);
  if (g.colscale >= 0) {
    const double sj = ((const double*)(sb + g.colscale))[j];
    v = sj > 0.0 ? cscale(v, 1.0 / sj) : make_double2(0.0, 0.0);
  }
  if (g.c0 >= 0) v = cadd(v, cscale(((const double2*)(sb + g.c0 + l * g.lc))[i * g.ldc + j], g.beta));
  C[i * g.ldc + j] = v;
}

// One refinement step of V (eigenvectors of H = Q^*Q) from T1 = V^*V (work3) and S = V^* H V
// (uq): lambda_i = s_ii / (1 - r_ii) with R = I - V^*V, the correction E with
// e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) (r_ij / 2 within a cluster of
// eigenvalues closer than delta = 2 (||S - diag(lambda)||_F + ||H||_F ||R||_F)), written as
// F = I + E into work4 for V <- V F; lambda into the sigma slots.  A step whose ||E||_F is at most
// 1e-9 (after the first) is the last one (state 2: its V F still runs; the next step marks the
// refinement converged, state 1): another would change V by less than the FP64 rounding of the
// products.
__global__ void __launch_bounds__(256) k_oa_step(Dev D, int iter) {
  __shared__ double s_red[32];
  __shared__ double s_lam[PRONY_MMAX];
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (!svd_live(p, st)) return;
  const int state = st.oa_conv;
  __syncthreads();
  if (state == 2 && threadIdx.x == 0) st.oa_conv = 1;
  if (state != 0) return;
  const int b = st.wv, LM = D.L.LDM;
  char* sb = D.small + p.soff;
  const double2* Hm = (const double2*)(sb + D.L.work1);
  const double2* T1 = (const double2*)(sb + D.L.work3);
  const double2* Sm = (const double2*)(sb + D.L.uq);
  double2* F = (double2*)(sb + D.L.work4);
  double* lam = (double*)(sb + D.L.sigma);
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
    s_lam[i] = Sm[i * LM + i].x / T1[i * LM + i].x;       // s_ii / (1 - r_ii), 1 - r_ii = (V^*V)_ii
    lam[i] = s_lam[i];
  }
  __syncthreads();
  double e1 = 0.0, e2 = 0.0, e3 = 0.0;
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int i = idx / b, j = idx % b;
    double2 sv = Sm[i * LM + j];
    if (i == j) sv.x -= s_lam[i];
    const double2 t = T1[i * LM + j];
    const double2 r = make_double2((i == j ? 1.0 : 0.0) - t.x, -t.y);
    e1 += cabs2(sv);
    e2 += cabs2(Hm[i * LM + j]);
    e3 += cabs2(r);
  }
  e1 = block_sum_d(e1, s_red);
  e2 = block_sum_d(e2, s_red);
  e3 = block_sum_d(e3, s_red);
  const double delta = 2.0 * (sqrt(e1) + sqrt(e2) * sqrt(e3));
  double en = 0.0;
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int i = idx / b, j = idx % b;
    const double2 t = T1[i * LM + j];
    const double2 r = make_double2((i == j ? 1.0 : 0.0) - t.x, -t.y);
    double2 e;
    if (i != j && fabs(s_lam[i] - s_lam[j]) > delta)
      e = cscale(cadd(Sm[i * LM + j], cscale(r, s_lam[j])), 1.0 / (s_lam[j] - s_lam[i]));
    else
      e = cscale(r, 0.5);
    en += cabs2(e);
    F[i * LM + j] = make_double2((i == j ? 1.0 : 0.0) + e.x, e.y);
  }
  en = block_sum_d(en, s_red);
  if (threadIdx.x == 0 && iter >= 1 && en <= 1e-18) st.oa_conv = 2;
}

// Eigenpairs of H in descending order: V_Q (vq) = the columns of the refined V (at byte offset
// `voff`) permuted, sigma = sqrt(lambda) sorted, sigma_m / sigma_1.
__global__ void __launch_bounds__(256) k_svd_sort(Dev D, long long voff) {
  __shared__ double s_lam[PRONY_MMAX];
  __shared__ int s_rank[PRONY_MMAX];
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (!svd_live(p, st)) return;
  const int b = st.wv, LM = D.L.LDM;
  char* sb = D.small + p.soff;
  const double2* Vm = (const double2*)(sb + voff);
  double2* VQ = (double2*)(sb + D.L.vq);
  double* sig = (double*)(sb + D.L.sigma);
  for (int i = threadIdx.x; i < b; i += blockDim.x) s_lam[i] = sig[i];
  __syncthreads();
  for (int j = threadIdx.x; j < b; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < b; ++i)
      if (s_lam[i] > s_lam[j] || (s_lam[i] == s_lam[j] && i < j)) ++r;
    s_rank[j] = r;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int i = idx / b, j = idx % b;
    VQ[i * LM + s_rank[j]] = Vm[i * LM + j];
  }
  for (int j = threadIdx.x; j < b; j += blockDim.x) sig[s_rank[j]] = sqrt(fmax(s_lam[j], 0.0));
  __syncthreads();
  if (threadIdx.x == 0) st.sigma_ratio = sig[0] > 0.0 ? sig[b - 1] / sig[0] : 0.0;
}

// z_j(l) = sum_a X[j][a] C_l[a][j] with X = W^{-1} (work3 after the Newton-Schulz steps) and
// C_l = S_l W (mproj slices); t_j(l) = -arg z_j(l) / 2 pi mod 1.
__global__ void k_eig_z(Dev D) {
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (!eig_live(p, st)) return;
  const int m = st.wv, LM = D.L.LDM, LR = D.L.LDR;
  char* sb = D.small + p.soff;
  const double2* Xd = (const double2*)(sb + D.L.work3);
  double* tout = (double*)(sb + D.L.t);
  double2* zr = (double2*)(sb + D.L.zraw);
  for (int q = threadIdx.x; q < m * p.d; q += blockDim.x) {
    const int j = q / p.d, l = q % p.d;
    const double2* Cl = (const double2*)(sb + D.L.mproj) + (size_t)l * LR * LM;
    double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int a = 0; a < m; ++a) acc[a & 3] = cadd(acc[a & 3], cmul(Xd[j * LM + a], Cl[a * LM + j]));
    const double2 z = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
    zr[j * PRONY_DMAX + l] = z;
    double tj = -atan2(z.y, z.x) / 6.283185307179586;
    tj -= floor(tj);
    if (tj >= 1.0) tj = 0.0;
    tout[j * PRONY_DMAX + l] = tj;
  }
  if (threadIdx.x == 0) st.rank_used = m;
}

// ----------------------------------------------------------------------------- SVD of Q and S_l
// FP32 one-sided Jacobi on the columns of Q: the starting V (FP64 copy in work2) of the FP64
// refinement.  One CTA per problem.
__global__ void __launch_bounds__(256) k_svd_jacobi(Dev D) {
  extern __shared__ float2 fsm[];
  __shared__ int s_rot;
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (!svd_live(p, st)) return;
  const int a = st.wu, b = st.wv;
  const int LM = D.L.LDM, LR = D.L.LDR;
  char* sb = D.small + p.soff;
  const double2* Q = (const double2*)(sb + D.L.q);            // a x b, ld LM
  double2* Vm = (double2*)(sb + D.L.work2);                     // b x b, ld LM
  float2* Qc = fsm;                                             // [b][a] columns (FP32)
  float2* Vc = fsm + (size_t)LM * LR;                           // [b][b] columns (FP32)

  // ---- FP32 one-sided Jacobi on the columns of Q
  for (int idx = threadIdx.x; idx < a * b; idx += blockDim.x) {
    int i = idx % a, j = idx / a;
    double2 q = Q[i * LM + j];
    Qc[j * a + i] = fc((float)q.x, (float)q.y);
  }
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    int i = idx % b, j = idx / b;
    Vc[j * b + i] = fc(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int nb = b + (b & 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const float jtol = 4.f * a * 5.9604645e-8f;
  const int max_sweeps = D.cap_jacobi > 0 ? D.cap_jacobi : 30;
  int sweep = 0;
  bool rotated = b > 1;                          // the last sweep still rotated (not converged)
  for (; sweep < max_sweeps && b > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step < nb - 1; ++step) {
      for (int k = warp; k < nb / 2; k += nwarp) {
        int pa, pb;
        rr_pair(step, k, nb, pa, pb);
        if (pa >= b || pb >= b) continue;
        if (pa > pb) { int t = pa; pa = pb; pb = t; }
        float al = 0.f, be = 0.f;
        float2 ga = fc(0.f, 0.f);
        for (int i = lane; i < a; i += 32) {
          float2 x = Qc[pa * a + i], y = Qc[pb * a + i];
          al += fabs2(x);
          be += fabs2(y);
          ga = fadd(ga, fmulc(x, y));
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
        }
        float ag = sqrtf(fabs2(ga));
        if (ag <= jtol * sqrtf(al * be) || ag == 0.f) continue;
        float zeta = (be - al) / (2.f * ag);
        float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        float c = rsqrtf(1.f + tt * tt), s = c * tt;
        float2 ph = fc(ga.x / ag, -ga.y / ag);   // e^{-i arg gamma}
        for (int i = lane; i < a; i += 32) {
          float2 x = Qc[pa * a + i], y = fmul(Qc[pb * a + i], ph);
          Qc[pa * a + i] = fsub(fscale(x, c), fscale(y, s));
          Qc[pb * a + i] = fadd(fscale(x, s), fscale(y, c));
        }
        for (int i = lane; i < b; i += 32) {
          float2 x = Vc[pa * b + i], y = fmul(Vc[pb * b + i], ph);
          Vc[pa * b + i] = fsub(fscale(x, c), fscale(y, s));
          Vc[pb * b + i] = fadd(fscale(x, s), fscale(y, c));
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    rotated = s_rot != 0;
    if (!s_rot) break;
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    int i = idx / b, j = idx % b;
    float2 v = Vc[j * b + i];
    Vm[i * LM + j] = make_double2(v.x, v.y);
  }
  if (threadIdx.x == 0) {
    st.oa_conv = 0;
    if (sweep >= max_sweeps && rotated) set_status_e(st, ST_ENOCONV);
  }
}

// Canonical phases: ph_j = v_j[argmax] / |.| of V_final = V V_Q (in B1); S_l <- D^* S_l D with
// D = diag(conj ph); U_Q, V_Q columns times conj(ph).
__global__ void k_canon(Dev D) {
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  const int b = st.wv, a = st.wu;
  if (st.done || b <= 0 || a <= 0 || b > p.m || a > p.r0) return;
  const int LM = D.L.LDM;
  __shared__ double2 ph[PRONY_MMAX];
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

// ----------------------------------------------------------------------------- eigen step
// C_mu, its eigenvectors W (FP32 Hessenberg reduction, shifted complex QR, triangular
// eigenvectors; FP64 copy in work2) and the FP32 Gauss-Jordan inverse X of W (FP64 copy in
// work3).  One CTA per problem.
__global__ void __launch_bounds__(256) k_eig_w(Dev D, unsigned long long seed) {
  extern __shared__ float2 esm[];
  __shared__ double2 mu[PRONY_DMAX];
  __shared__ float2 hv[PRONY_MMAX];
  __shared__ float2 sv[PRONY_MMAX];
  __shared__ float s_norm;
  __shared__ int s_fail, s_pr;
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (!eig_live(p, st)) return;                 // shared memory holds 3 maxM^2 entries
  const int m = st.wv;
  const int LM = D.L.LDM;
  const int LD = m;                             // smem leading dimension
  float2* H = esm;                              // m x m  (C_mu, then Schur form, then W^{-1} work)
  float2* Z = esm + LD * LD;                    // m x m  (Schur vectors, then W)
  float2* Y = Z + LD * LD;                      // m x m  (triangular eigenvectors, then W^{-1})
  char* sb = D.small + p.soff;
  const double2* S = (const double2*)(sb + D.L.S);
  double2* Wd = (double2*)(sb + D.L.work2);     // W (FP64)
  double2* Xd = (double2*)(sb + D.L.work3);     // W^{-1} (FP64, FP32 accurate)
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
    for (int l = 0; l < p.d; ++l) acc = cadd(acc, cmul(mu[l], S[(size_t)l * LM * LM + i * LM + j]));
    H[i * LD + j] = fc((float)acc.x, (float)acc.y);
    Z[i * LD + j] = fc(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // ---- FP32 Householder reduction to Hessenberg form
  for (int k = 0; k + 2 < m; ++k) {
    if (threadIdx.x == 0) {
      float nx = 0.f;
      for (int i = k + 1; i < m; ++i) nx += fabs2(H[i * LD + k]);
      nx = sqrtf(nx);
      float2 x0 = H[(k + 1) * LD + k];
      float ax0 = sqrtf(fabs2(x0));
      float2 ph = ax0 > 0.f ? fscale(x0, 1.f / ax0) : fc(1.f, 0.f);
      float2 alpha = fscale(ph, -nx);
      for (int i = 0; i < m; ++i) hv[i] = fc(0.f, 0.f);
      for (int i = k + 1; i < m; ++i) hv[i] = H[i * LD + k];
      hv[k + 1] = fsub(hv[k + 1], alpha);
      float nv = 0.f;
      for (int i = k + 1; i < m; ++i) nv += fabs2(hv[i]);
      s_norm = nv;
      if (nv > 0.f) {
        float inv = rsqrtf(nv);
        for (int i = k + 1; i < m; ++i) hv[i] = fscale(hv[i], inv);
      }
    }
    __syncthreads();
    if (s_norm > 0.f) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        float2 s = fc(0.f, 0.f);
        for (int i = k + 1; i < m; ++i) s = fadd(s, fmulc(hv[i], H[i * LD + j]));
        sv[j] = s;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < (m - k - 1) * m; idx += blockDim.x) {
        int i = k + 1 + idx / m, j = idx % m;
        H[i * LD + j] = fsub(H[i * LD + j], fscale(fmul(hv[i], sv[j]), 2.f));
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
        float2* R = i < m ? H : Z;
        int ii = i < m ? i : i - m;
        float2 s = fc(0.f, 0.f);
        for (int j = k + 1; j < m; ++j) s = fadd(s, fmul(R[ii * LD + j], hv[j]));
        for (int j = k + 1; j < m; ++j) R[ii * LD + j] = fsub(R[ii * LD + j], fscale(fmul(s, fconj(hv[j])), 2.f));
      }
      __syncthreads();
      for (int i = k + 2 + threadIdx.x; i < m; i += blockDim.x) H[i * LD + k] = fc(0.f, 0.f);
      __syncthreads();
    }
  }
  // ---- FP32 shifted complex QR iteration (one warp), full Schur form
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const float eps = 5.9604645e-8f;
    int hi = m - 1, its = 0, total = 0;
    const int cap = D.cap_eigqr > 0 ? D.cap_eigqr : 30 * m + 30;
    while (hi > 0) {
      if (total > cap) break;
      int l = hi;
      for (; l > 0; --l) {
        float s = fabs1(H[(l - 1) * LD + l - 1]) + fabs1(H[l * LD + l]);
        if (s == 0.f) s = 1.f;
        if (fabs1(H[l * LD + l - 1]) <= eps * s) break;
      }
      if (l > 0 && lane == 0) H[l * LD + l - 1] = fc(0.f, 0.f);
      __syncwarp();
      if (l == hi) {
        --hi;
        its = 0;
        continue;
      }
      float2 sh;
      if (its == 10 || its == 20) {
        sh = fadd(H[hi * LD + hi], fc(0.75f * fabs1(H[hi * LD + hi - 1]), 0.f));
      } else {
        float2 a = H[(hi - 1) * LD + hi - 1], bb = H[(hi - 1) * LD + hi], c = H[hi * LD + hi - 1], dd = H[hi * LD + hi];
        float2 hd = fscale(fsub(a, dd), 0.5f);
        float2 disc = fsqrtc(fadd(fmul(hd, hd), fmul(bb, c)));
        float2 mid = fscale(fadd(a, dd), 0.5f);
        float2 l1 = fadd(mid, disc), l2 = fsub(mid, disc);
        sh = fabs2(fsub(l1, dd)) <= fabs2(fsub(l2, dd)) ? l1 : l2;
      }
      float2 x = fsub(H[l * LD + l], sh), y = H[(l + 1) * LD + l];
      for (int k = l; k < hi; ++k) {
        if (k > l) {
          x = H[k * LD + k - 1];
          y = H[(k + 1) * LD + k - 1];
        }
        float ax = sqrtf(fabs2(x)), ay = sqrtf(fabs2(y));
        float nr = hypotf(ax, ay);
        float c;
        float2 s;
        if (nr == 0.f) {
          c = 1.f;
          s = fc(0.f, 0.f);
        } else if (ax == 0.f) {
          c = 0.f;
          s = fscale(fconj(y), 1.f / ay);
        } else {
          c = ax / nr;
          s = fscale(fmul(fscale(x, 1.f / ax), fconj(y)), 1.f / nr);
        }
        for (int j = max(l, k - 1) + lane; j < m; j += 32) {
          float2 rk = H[k * LD + j], rk1 = H[(k + 1) * LD + j];
          H[k * LD + j] = fadd(fscale(rk, c), fmul(s, rk1));
          H[(k + 1) * LD + j] = fsub(fscale(rk1, c), fmul(fconj(s), rk));
        }
        __syncwarp();
        int rmax = min(k + 2, hi);
        for (int i = lane; i <= rmax; i += 32) {
          float2 ck = H[i * LD + k], ck1 = H[i * LD + k + 1];
          H[i * LD + k] = fadd(fscale(ck, c), fmul(fconj(s), ck1));
          H[i * LD + k + 1] = fsub(fscale(ck1, c), fmul(s, ck));
        }
        for (int i = lane; i < m; i += 32) {
          float2 ck = Z[i * LD + k], ck1 = Z[i * LD + k + 1];
          Z[i * LD + k] = fadd(fscale(ck, c), fmul(fconj(s), ck1));
          Z[i * LD + k + 1] = fsub(fscale(ck1, c), fmul(s, ck));
        }
        __syncwarp();
      }
      ++its;
      ++total;
    }
    if (lane == 0 && hi > 0) s_fail = 1;
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0) set_status_e(st, ST_ENOCONV);
  // ---- triangular eigenvectors (FP32), W = Z Y with unit columns
  if (threadIdx.x == 0) {
    float hn = 0.f;
    for (int i = 0; i < m; ++i)
      for (int j = i; j < m; ++j) hn = fmaxf(hn, fabs1(H[i * LD + j]));
    s_norm = hn;
  }
  __syncthreads();
  const float small = fmaxf(s_norm, 1e-30f) * 5.9604645e-8f;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    float2 lam = H[k * LD + k];
    for (int i = k + 1; i < m; ++i) Y[i * LD + k] = fc(0.f, 0.f);
    Y[k * LD + k] = fc(1.f, 0.f);
    for (int i = k - 1; i >= 0; --i) {
      float2 s = fc(0.f, 0.f);
      for (int j = i + 1; j <= k; ++j) s = fadd(s, fmul(H[i * LD + j], Y[j * LD + k]));
      float2 den = fsub(H[i * LD + i], lam);
      if (fabs1(den) < small) den = fc(small, 0.f);
      Y[i * LD + k] = fdiv(fc(-s.x, -s.y), den);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, k = idx % m;
    float2 acc = fc(0.f, 0.f);
    for (int j = 0; j <= k; ++j) acc = fadd(acc, fmul(Z[i * LD + j], Y[j * LD + k]));
    H[i * LD + k] = acc;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < m; ++i) s += fabs2(H[i * LD + k]);
    sv[k] = fc(s > 0.f ? rsqrtf(s) : 1.f, 0.f);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, k = idx % m;
    float2 w = fscale(H[i * LD + k], sv[k].x);
    Z[i * LD + k] = w;                                  // W (FP32) for the inverse
    Wd[i * LM + k] = make_double2(w.x, w.y);            // W (FP64, exactly the same numbers)
    Y[i * LD + k] = fc(i == k ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // ---- FP32 Gauss-Jordan inverse of W (partial pivoting): Z -> I, Y -> W^{-1}
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      int pr = k;
      float best = fabs1(Z[k * LD + k]);
      for (int i = k + 1; i < m; ++i) {
        float v = fabs1(Z[i * LD + k]);
        if (v > best) { best = v; pr = i; }
      }
      s_pr = pr;
      if (best == 0.f) s_fail = 2;
    }
    __syncthreads();
    const int pr = s_pr;
    if (pr != k) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        float2 t = Z[k * LD + j]; Z[k * LD + j] = Z[pr * LD + j]; Z[pr * LD + j] = t;
        t = Y[k * LD + j]; Y[k * LD + j] = Y[pr * LD + j]; Y[pr * LD + j] = t;
      }
      __syncthreads();
    }
    float2 piv = Z[k * LD + k];
    if (fabs1(piv) == 0.f) piv = fc(1e-30f, 0.f);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      Z[k * LD + j] = fdiv(Z[k * LD + j], piv);
      Y[k * LD + j] = fdiv(Y[k * LD + j], piv);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) hv[i] = (i == k) ? fc(0.f, 0.f) : Z[i * LD + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = idx / m, j = idx % m;
      if (i == k) continue;
      float2 f = hv[i];
      Z[i * LD + j] = fsub(Z[i * LD + j], fmul(f, Z[k * LD + j]));
      Y[i * LD + j] = fsub(Y[i * LD + j], fmul(f, Y[k * LD + j]));
    }
    __syncthreads();
  }  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    float2 x = Y[i * LD + j];
    Xd[i * LM + j] = make_double2(x.x, x.y);
  }
  if (threadIdx.x == 0 && s_fail == 2) set_status_e(st, ST_ENOCONV);
}

}  // namespace

namespace {
constexpr int OA_MAX = 4;     // refinement steps launched (converged problems skip the rest)

void launch_zgemm(const Dev& D, const ZG& g, cudaStream_t s) {
  // tiles of the largest product of the batch: widths are at most r0 (a) and m (b)
  const int mx = g.M == ZD_A ? D.L.LDR : D.L.LDM, nx = g.N == ZD_A ? D.L.LDR : D.L.LDM;
  const int tiles = ((mx + ZT - 1) / ZT) * ((nx + ZT - 1) / ZT);
  note_launch();
  k_zgemm<<<dim3(tiles, D.nprob, g.nl), ZT * ZT, 0, s>>>(D, g);
}

ZG zg(long long a, int lda, int ta, long long b, int ldb, int tb, long long c, int ldc, int M, int N, int K,
      int live) {
  ZG g{};
  g.a = a; g.b = b; g.c = c; g.c0 = -1;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.ta = ta; g.tb = tb;
  g.M = M; g.N = N; g.K = K;
  g.nl = 1;
  g.colscale = -1;
  g.live = live;
  g.conv = ZC_ALL;
  g.alpha = 1.0;
  g.beta = 0.0;
  return g;
}
}  // namespace

void launch_svd_S(const Dev& D, cudaStream_t s) {
  static size_t set = 0;
  const SmallLay& L = D.L;
  const int LM = L.LDM;
  size_t sm = sizeof(float2) * ((size_t)L.LDM * L.LDR + (size_t)L.LDM * L.LDM);
  if (sm > set) {
    cudaFuncSetAttribute(k_svd_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set = sm;
  }
  // H = Q^* Q (work1); starting V (work2) by FP32 Jacobi
  launch_zgemm(D, zg(L.q, LM, 1, L.q, LM, 0, L.work1, LM, ZD_B, ZD_B, ZD_A, ZL_SVD), s);
  note_launch();
  k_svd_jacobi<<<D.nprob, 256, sm, s>>>(D);
  // refinement steps; V alternates between work2 and the first S_l slot (free until the end)
  long long v = L.work2, vn = L.S;
  for (int it = 0; it < OA_MAX; ++it) {
    ZG t1 = zg(v, LM, 1, v, LM, 0, L.work3, LM, ZD_B, ZD_B, ZD_B, ZL_SVD);   // V^* V
    t1.conv = ZC_SKIP_CONV;
    launch_zgemm(D, t1, s);
    ZG t2 = zg(L.work1, LM, 0, v, LM, 0, L.work4, LM, ZD_B, ZD_B, ZD_B, ZL_SVD);   // H V
    t2.conv = ZC_SKIP_CONV;
    launch_zgemm(D, t2, s);
    ZG sv = zg(v, LM, 1, L.work4, LM, 0, L.uq, LM, ZD_B, ZD_B, ZD_B, ZL_SVD);   // V^* H V
    sv.conv = ZC_SKIP_CONV;
    launch_zgemm(D, sv, s);
    note_launch();
    k_oa_step<<<D.nprob, 256, 0, s>>>(D, it);
    ZG vf = zg(v, LM, 0, L.work4, LM, 0, vn, LM, ZD_B, ZD_B, ZD_B, ZL_SVD);   // V F
    vf.conv = ZC_COPY_CONV;
    launch_zgemm(D, vf, s);
    std::swap(v, vn);
  }
  note_launch();
  k_svd_sort<<<D.nprob, 256, 0, s>>>(D, v);
  // U_Q = Q V_Q Sigma^{-1} (a x b)
  ZG uq = zg(L.q, LM, 0, L.vq, LM, 0, L.uq, LM, ZD_A, ZD_B, ZD_B, ZL_SVD);
  uq.colscale = L.sigma;
  launch_zgemm(D, uq, s);
  // P_l = U_Q^* M_l (b x b, into work1 + l (work2 - work1)); S_l = P_l V_Q Sigma^{-1}
  ZG pl = zg(L.uq, LM, 1, L.mproj, LM, 0, L.work1, LM, ZD_B, ZD_B, ZD_A, ZL_SVD);
  pl.nl = D.maxD;
  pl.lb = 16LL * L.LDR * L.LDM;
  pl.lc = L.work2 - L.work1;
  launch_zgemm(D, pl, s);
  ZG sl = zg(L.work1, LM, 0, L.vq, LM, 0, L.S, LM, ZD_B, ZD_B, ZD_B, ZL_SVD);
  sl.nl = D.maxD;
  sl.la = L.work2 - L.work1;
  sl.lc = 16LL * L.LDM * L.LDM;
  sl.colscale = L.sigma;
  launch_zgemm(D, sl, s);
}

void launch_canon(const Dev& D, cudaStream_t s) {
  note_launch();
  k_canon<<<D.nprob, 256, 0, s>>>(D);
}

void launch_eig_t(const Dev& D, unsigned long long seed, cudaStream_t s) {
  static size_t set = 0;
  const SmallLay& L = D.L;
  const int LM = L.LDM;
  size_t sm = sizeof(float2) * 3 * (size_t)D.maxM * D.maxM;
  if (sm > set) {
    cudaFuncSetAttribute(k_eig_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(sm, 1024));
    set = sm;
  }
  note_launch();
  k_eig_w<<<D.nprob, 256, std::max<size_t>(sm, 16), s>>>(D, seed);
  // two Newton-Schulz steps X <- 2X - X (W X): W in work2, X in work3 -> work1 -> work3
  long long x = L.work3, xn = L.work1;
  for (int it = 0; it < 2; ++it) {
    launch_zgemm(D, zg(L.work2, LM, 0, x, LM, 0, L.work4, LM, ZD_B, ZD_B, ZD_B, ZL_EIG), s);   // R = W X
    ZG ns = zg(x, LM, 0, L.work4, LM, 0, xn, LM, ZD_B, ZD_B, ZD_B, ZL_EIG);                  // 2X - X R
    ns.alpha = -1.0;
    ns.c0 = x;
    ns.beta = 2.0;
    launch_zgemm(D, ns, s);
    std::swap(x, xn);
  }
  // C_l = S_l W into the mproj slices, then z and t
  ZG cl = zg(L.S, LM, 0, L.work2, LM, 0, L.mproj, LM, ZD_B, ZD_B, ZD_B, ZL_EIG);
  cl.nl = D.maxD;
  cl.la = 16LL * L.LDM * L.LDM;
  cl.lc = 16LL * L.LDR * L.LDM;
  launch_zgemm(D, cl, s);
  note_launch();
  k_eig_z<<<D.nprob, 128, 0, s>>>(D);
}
