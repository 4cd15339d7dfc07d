// Least-squares refinement of the exponential-sum parameters (t_j, c_j) by damped Gauss-Newton
// (Levenberg-Marquardt) steps on L(t, c) = sum_k |f(k; t, c) - y_k|^2, f from Eq. (1), over an
// integer box of sample points.  Every step runs on the device:
//   k_lm_normal  one pass over the points: residual r_k, L, and the weighted Grams
//                M^{ll'}_{ab} = sum_k w_l(k) w_l'(k) conj(e_ak) e_bk  (w_0 = 1, w_l = k_l)
//                V^{l}_a      = sum_k w_l(k) conj(e_ak) r_k,
//                from which J^* J and J^* r of the real parameter vector follow in closed form
//   k_lm_solve   one CTA: the real normal equations Re(J^*J) delta = -Re(J^*r) with Marquardt
//                damping, Jacobi-scaled and solved by an FP32 Cholesky factorisation
//   k_lm_trial   the loss at the candidate parameters
//   k_lm_update  accept (loss decreased) or reject, adapt the damping, clear the accumulators
// The exponentials are recomputed in every pass, never stored; phases <t_j, k> mod 1 are exact
// 64-bit fixed-point sums, the exponentials and sums FP32 per CTA, the accumulators FP64.
#include "common.cuh"

#include <algorithm>

namespace {

constexpr int LM_TILE = 128;            // points per CTA (= threads) in the point passes
constexpr double TWO_PI = 6.283185307179586;

__device__ inline int combo(int l, int lp, int d) {      // index of the pair l <= lp in {0..d}
  if (l > lp) { int x = l; l = lp; lp = x; }
  return l * (d + 1) - l * (l - 1) / 2 + (lp - l);
}

// Residual r_k = f(k) - y_k at the point of thread `i` of a tile, with its exponentials in E.
__device__ inline float2 point_residual(const uint64_t* T, const float2* cs, int m, int d, const Box& B,
                                        long long q, long long K, const float2* y, float2* E, int ldE, int* k) {
  if (q >= K) {
    for (int j = 0; j < m; ++j) E[j * ldE] = make_float2(0.f, 0.f);
    for (int l = 0; l < d; ++l) k[l] = 0;
    return make_float2(0.f, 0.f);
  }
  box_point(B, d, q, k);
  float2 f = make_float2(0.f, 0.f);
  for (int j = 0; j < m; ++j) {
    const float u = centred_phase(T + j * d, k, d);
    float sn, cn;
    sincospif(2.0f * u, &sn, &cn);                 // e = exp(-2 pi i u) = cn - i sn
    E[j * ldE] = make_float2(cn, -sn);
    f.x += cs[j].x * cn + cs[j].y * sn;
    f.y += cs[j].y * cn - cs[j].x * sn;
  }
  const float2 yk = y[q];
  return make_float2(f.x - yk.x, f.y - yk.y);
}

__device__ inline float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

__device__ inline void load_params(const double* t, const double2* c, int m, int d, uint64_t* T, float2* cs) {
  for (int q = threadIdx.x; q < m * d; q += blockDim.x) T[q] = frac64(t[q]);
  for (int q = threadIdx.x; q < m; q += blockDim.x) cs[q] = make_float2((float)c[q].x, (float)c[q].y);
}

// acc layout (double2): M[NC][m][m], V[d+1][m]; then loss, loss_trial (double)
template <int d>
__global__ void __launch_bounds__(LM_TILE) k_lm_normal(const double* t, const double2* c, int m, Box B, long long K,
                                                       const float2* y, double2* M, double2* V, double* loss) {
  extern __shared__ float2 lm_smem[];
  float2* E = lm_smem;                                   // m x LM_TILE
  float2* R = E + m * LM_TILE;                           // LM_TILE
  float* Wt = (float*)(R + LM_TILE);                     // d x LM_TILE
  __shared__ uint64_t T[PRONY_MMAX * PRONY_DMAX];
  __shared__ float2 cs[PRONY_MMAX];
  __shared__ float red[LM_TILE / 32];
  load_params(t, c, m, d, T, cs);
  __syncthreads();
  const int i = threadIdx.x;
  const long long q = blockIdx.x * (long long)LM_TILE + i;
  int k[PRONY_DMAX];
  const float2 r = point_residual(T, cs, m, d, B, q, K, y, E + i, LM_TILE, k);
  R[i] = r;
  for (int l = 0; l < d; ++l) Wt[l * LM_TILE + i] = (float)k[l];
  const float l2 = block_sum(r.x * r.x + r.y * r.y, red);
  if (i == 0) atomicAdd(loss, (double)l2);
  __syncthreads();
  constexpr int NC = (d + 1) * (d + 2) / 2;
  const long long left = K - blockIdx.x * (long long)LM_TILE;
  const int npt = left < LM_TILE ? (int)left : LM_TILE;
  for (int idx = i; idx < m * m; idx += LM_TILE) {
    const int a = idx / m, b = idx % m;
    float2 acc[NC];
#pragma unroll
    for (int x = 0; x < NC; ++x) acc[x] = make_float2(0.f, 0.f);
    for (int p = 0; p < npt; ++p) {
      const float2 ea = E[a * LM_TILE + p], eb = E[b * LM_TILE + p];
      const float2 pr = make_float2(ea.x * eb.x + ea.y * eb.y, ea.x * eb.y - ea.y * eb.x);   // conj(ea) eb
      acc[0].x += pr.x;
      acc[0].y += pr.y;
      float wk[d];
#pragma unroll
      for (int l = 0; l < d; ++l) wk[l] = Wt[l * LM_TILE + p];
#pragma unroll
      for (int l = 1; l <= d; ++l) {
        acc[l].x += wk[l - 1] * pr.x;                      // (0, l)
        acc[l].y += wk[l - 1] * pr.y;
      }
      int x = d + 1;
#pragma unroll
      for (int l = 1; l <= d; ++l)
#pragma unroll
        for (int lp = l; lp <= d; ++lp, ++x) {
          const float w2 = wk[l - 1] * wk[lp - 1];
          acc[x].x += w2 * pr.x;
          acc[x].y += w2 * pr.y;
        }
    }
    // accumulator order above: (0,0), (0,1..d), then (l, lp >= l) for l >= 1 -- the order of combo()
#pragma unroll
    for (int x = 0; x < NC; ++x) {
      double2* dst = M + ((long long)x * m + a) * m + b;
      atomicAdd(&dst->x, (double)acc[x].x);
      atomicAdd(&dst->y, (double)acc[x].y);
    }
  }
  for (int idx = i; idx < m * (d + 1); idx += LM_TILE) {
    const int a = idx % m, l = idx / m;
    float2 acc = make_float2(0.f, 0.f);
    for (int p = 0; p < npt; ++p) {
      const float2 ea = E[a * LM_TILE + p], rp = R[p];
      const float w = l == 0 ? 1.f : Wt[(l - 1) * LM_TILE + p];
      acc.x += w * (ea.x * rp.x + ea.y * rp.y);            // conj(ea) r
      acc.y += w * (ea.x * rp.y - ea.y * rp.x);
    }
    double2* dst = V + (long long)l * m + a;
    atomicAdd(&dst->x, (double)acc.x);
    atomicAdd(&dst->y, (double)acc.y);
  }
}

__global__ void __launch_bounds__(LM_TILE) k_lm_trial(const double* t, const double2* c, int m, int d, Box B,
                                                      long long K, const float2* y, double* loss) {
  extern __shared__ float2 lm_smem[];
  __shared__ uint64_t T[PRONY_MMAX * PRONY_DMAX];
  __shared__ float2 cs[PRONY_MMAX];
  __shared__ float red[LM_TILE / 32];
  load_params(t, c, m, d, T, cs);
  __syncthreads();
  const long long q = blockIdx.x * (long long)LM_TILE + threadIdx.x;
  int k[PRONY_DMAX];
  const float2 r = point_residual(T, cs, m, d, B, q, K, y, lm_smem + threadIdx.x, LM_TILE, k);
  const float l2 = block_sum(r.x * r.x + r.y * r.y, red);
  if (threadIdx.x == 0) atomicAdd(loss, (double)l2);
}

struct LmState {
  double lambda;
  int accepted;
};

// sigma_alpha(a): the factor of column (a, alpha) of J besides w_{lambda(alpha)}(k) e_ak.
// alpha < d: t_a(alpha) -> -2 pi i c_a, weight index alpha + 1;  alpha = d: Re c_a -> 1;  d + 1: Im c_a -> i.
__device__ inline double2 sigma_of(int alpha, int d, double2 ca, int& widx) {
  if (alpha < d) {
    widx = alpha + 1;
    return make_double2(TWO_PI * ca.y, -TWO_PI * ca.x);
  }
  widx = 0;
  return alpha == d ? make_double2(1.0, 0.0) : make_double2(0.0, 1.0);
}

// One CTA: damped normal equations -> candidate (tc, cc).  P = m (d + 2) real parameters.
__global__ void __launch_bounds__(256) k_lm_solve(const double* t, const double2* c, int m, int d, const double2* M,
                                                  const double2* V, const LmState* st, double* tc, double2* cc) {
  extern __shared__ float lm_f[];
  const int P = m * (d + 2);
  float* A = lm_f;                                   // P x P (lower triangle used), Jacobi-scaled
  float* g = A + P * P;                              // P
  float* sc = g + P;                                 // P: 1 / sqrt(damped diagonal)
  const double lam = st->lambda;
  // diagonal first (for the scaling)
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const int a = p / (d + 2), al = p % (d + 2);
    int wi;
    const double2 s = sigma_of(al, d, c[a], wi);
    const double2 Mv = M[((long long)combo(wi, wi, d) * m + a) * m + a];
    const double diag = (s.x * s.x + s.y * s.y) * Mv.x;
    const double dd = diag * (1.0 + lam) + 1e-30;
    sc[p] = (float)(1.0 / sqrt(dd));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < P * P; idx += blockDim.x) {
    const int p = idx / P, q = idx % P;
    if (q > p) continue;
    const int a = p / (d + 2), al = p % (d + 2), b = q / (d + 2), be = q % (d + 2);
    int wa, wb;
    const double2 sa = sigma_of(al, d, c[a], wa), sb = sigma_of(be, d, c[b], wb);
    const double2 Mv = M[((long long)combo(wa, wb, d) * m + a) * m + b];
    // Re( conj(sa) sb M )
    const double2 ss = make_double2(sa.x * sb.x + sa.y * sb.y, sa.x * sb.y - sa.y * sb.x);
    double v = ss.x * Mv.x - ss.y * Mv.y;
    if (p == q) v *= (1.0 + lam);
    A[p * P + q] = (float)(v * (double)sc[p] * (double)sc[q]);
  }
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const int a = p / (d + 2), al = p % (d + 2);
    int wi;
    const double2 s = sigma_of(al, d, c[a], wi);
    const double2 v = V[(long long)wi * m + a];
    const double re = s.x * v.x + s.y * v.y;          // Re( conj(s) v )
    g[p] = (float)(-re * (double)sc[p]);
  }
  __syncthreads();
  // Cholesky A = L L^T (lower, in place), right-looking
  for (int j = 0; j < P; ++j) {
    if (threadIdx.x == 0) A[j * P + j] = sqrtf(fmaxf(A[j * P + j], 1e-20f));
    __syncthreads();
    const float ljj = A[j * P + j];
    for (int i = j + 1 + threadIdx.x; i < P; i += blockDim.x) A[i * P + j] /= ljj;
    __syncthreads();
    const int rem = P - j - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int i = j + 1 + idx / rem, k2 = j + 1 + idx % rem;
      if (k2 <= i) A[i * P + k2] -= A[i * P + j] * A[k2 * P + j];
    }
    __syncthreads();
  }
  // triangular solves by one warp: L z = g, L^T x = z
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int j = 0; j < P; ++j) {
      const float zj = g[j] / A[j * P + j];
      __syncwarp();
      for (int i = j + 1 + lane; i < P; i += 32) g[i] -= A[i * P + j] * zj;
      if (lane == 0) g[j] = zj;
      __syncwarp();
    }
    for (int j = P - 1; j >= 0; --j) {
      const float xj = g[j] / A[j * P + j];
      __syncwarp();
      for (int i = lane; i < j; i += 32) g[i] -= A[j * P + i] * xj;
      if (lane == 0) g[j] = xj;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const int a = p / (d + 2), al = p % (d + 2);
    const double delta = (double)g[p] * (double)sc[p];
    if (al < d) {
      double v = t[a * d + al] + delta;
      v -= floor(v);                                   // f is 1-periodic in each t_a(l)
      tc[a * d + al] = v;
    } else if (al == d) {
      cc[a].x = c[a].x + delta;
    } else {
      cc[a].y = c[a].y + delta;
    }
  }
}

// Accept or reject the candidate; record the loss; clear the accumulators of the next step.
__global__ void k_lm_update(double* t, double2* c, const double* tc, const double2* cc, int m, int d,
                            LmState* st, double2* acc, long long nacc, double* loss, double* hist, int it) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const double l0 = loss[0], l1 = loss[1];
    ok = (l1 < l0 && isfinite(l1)) ? 1 : 0;
    if (hist) {
      hist[it] = l0;
      hist[it + 1] = ok ? l1 : l0;
    }
    st->lambda = ok ? fmax(st->lambda * (1.0 / 3.0), 1e-12) : fmin(st->lambda * 4.0, 1e12);
    st->accepted += ok;
  }
  __syncthreads();
  if (ok) {
    for (int q = threadIdx.x; q < m * d; q += blockDim.x) t[q] = tc[q];
    for (int q = threadIdx.x; q < m; q += blockDim.x) c[q] = cc[q];
  }
  for (long long q = threadIdx.x; q < nacc; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
  if (threadIdx.x < 2) loss[threadIdx.x] = 0.0;
}

__global__ void k_lm_init(LmState* st, double lambda0, double2* acc, long long nacc, double* loss, const double2* c,
                          double2* cc, int m) {
  if (threadIdx.x == 0) {
    st->lambda = lambda0;
    st->accepted = 0;
  }
  for (long long q = threadIdx.x; q < nacc; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
  for (int q = threadIdx.x; q < m; q += blockDim.x) cc[q] = c[q];
  if (threadIdx.x < 2) loss[threadIdx.x] = 0.0;
}

inline int lm_blocks(long long K) { return (int)((K + LM_TILE - 1) / LM_TILE); }

}  // namespace

// ----------------------------------------------------------------------------- host side
long long lm_workspace_bytes(int m, int d) {
  const int NC = (d + 1) * (d + 2) / 2;
  const long long nacc = (long long)NC * m * m + (long long)(d + 1) * m;
  return 16 * nacc + 16 * m + 8 * (long long)m * d + 16 + 64;
}

size_t lm_solve_smem(int m, int d) {
  const int P = m * (d + 2);
  return sizeof(float) * ((size_t)P * P + 2 * P);
}

static size_t lm_normal_smem(int m, int d) {
  return sizeof(float2) * (size_t)(m + 1) * LM_TILE + sizeof(float) * (size_t)d * LM_TILE;
}

// Dynamic shared-memory limits of the refinement kernels (outside any stream capture).
cudaError_t lm_set_attributes(int m, int d) {
  static size_t set_n[PRONY_DMAX + 1] = {0, 0, 0, 0, 0}, set_t = 0, set_s = 0;
  void (*normal)(const double*, const double2*, int, Box, long long, const float2*, double2*, double2*, double*) =
      d == 1 ? k_lm_normal<1> : d == 2 ? k_lm_normal<2> : d == 3 ? k_lm_normal<3> : k_lm_normal<4>;
  const size_t sn = lm_normal_smem(m, d), st = sizeof(float2) * (size_t)m * LM_TILE, ss = lm_solve_smem(m, d);
  cudaError_t e = cudaSuccess;
  if (sn > set_n[d] && (e = cudaFuncSetAttribute(normal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sn)) ==
                           cudaSuccess)
    set_n[d] = sn;
  if (e == cudaSuccess && st > set_t &&
      (e = cudaFuncSetAttribute(k_lm_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st)) == cudaSuccess)
    set_t = st;
  if (e == cudaSuccess && ss > set_s &&
      (e = cudaFuncSetAttribute(k_lm_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss)) == cudaSuccess)
    set_s = ss;
  return e;
}

// The whole refinement, enqueued on `s` (launches only: capturable in a CUDA graph; the
// shared-memory attributes are set beforehand by lm_set_attributes).
void launch_refine_lm(double* t, double2* c, int m, int d, const int* lo, const int* len, long long K,
                      const float2* y, int iters, double lambda0, double* hist, void* ws, cudaStream_t s) {
  const int NC = (d + 1) * (d + 2) / 2;
  const long long nacc = (long long)NC * m * m + (long long)(d + 1) * m;
  double2* acc = (double2*)ws;
  double2* M = acc;
  double2* V = acc + (long long)NC * m * m;
  double2* cc = acc + nacc;
  double* tc = (double*)(cc + m);
  double* loss = tc + m * d;                            // loss, loss_trial
  LmState* st = (LmState*)(loss + 2);
  const Box B = make_box(d, lo, len);
  const size_t sm_normal = lm_normal_smem(m, d);
  const size_t sm_trial = sizeof(float2) * (size_t)m * LM_TILE;
  const size_t sm_solve = lm_solve_smem(m, d);
  void (*normal)(const double*, const double2*, int, Box, long long, const float2*, double2*, double2*, double*) =
      d == 1 ? k_lm_normal<1> : d == 2 ? k_lm_normal<2> : d == 3 ? k_lm_normal<3> : k_lm_normal<4>;
  note_launch();
  k_lm_init<<<1, 256, 0, s>>>(st, lambda0, acc, nacc, loss, c, cc, m);
  for (int it = 0; it < iters; ++it) {
    note_launch();
    normal<<<lm_blocks(K), LM_TILE, sm_normal, s>>>(t, c, m, B, K, y, M, V, loss);
    note_launch();
    k_lm_solve<<<1, 256, sm_solve, s>>>(t, c, m, d, M, V, st, tc, cc);
    note_launch();
    k_lm_trial<<<lm_blocks(K), LM_TILE, sm_trial, s>>>(tc, cc, m, d, B, K, y, loss + 1);
    note_launch();
    k_lm_update<<<1, 256, 0, s>>>(t, c, tc, cc, m, d, st, acc, nacc, loss, hist, it);
  }
}
