// Lanczos bidiagonalisation with full reorthogonalisation (Algorithm 2, Section 2.1), batched:
// every launch advances every problem that has not stopped by one half step.  Vectors live in
// the tall blocks V (v_0 .. v_k) and U (u_0 .. u_{k-1}); the Toeplitz products of a single column
// use the same kernels as the block power method (column in B1, result in B2); the
// reorthogonalisation against all previous vectors is classical Gram-Schmidt applied twice
// (coefficients by the tall-skinny Gram, update by the X M kernel).  A problem stops when alpha
// or beta falls below tol ||T||_F (the rank it reveals is the number of accepted u), or when the
// basis fills the r0 columns of its blocks.
#include "common.cuh"

#include <algorithm>

namespace {

__device__ inline float2* lz_col(const Dev& D, int buf, const ProbDesc& p, int col) {
  float2* base = buf == BUF_U ? D.U : buf == BUF_V ? D.V : buf == BUF_B1 ? D.B1 : D.B2;
  return base + p.xoff + (long long)col * p.N;
}

__device__ inline float block_sum_f(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;   // every thread
}

// v_0 = first column of the random start block, normalised; k = 0.
__global__ void k_lz_start(Dev D) {
  __shared__ float sh[32];
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (st.done) return;
  float2* v = lz_col(D, BUF_V, p, 0);
  float acc = 0.f;
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) acc += v[i].x * v[i].x + v[i].y * v[i].y;
  const float nrm = sqrtf(block_sum_f(acc, sh));
  const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) v[i] = make_float2(v[i].x * inv, v[i].y * inv);
  if (threadIdx.x == 0) {
    st.lk = 0;
    st.lstop = 0;
    st.lalpha = 0.0;
    st.lbeta = 0.0;
  }
}

// B1[:, 0] = v_k (which = 0) or u_k (which = 1).
__global__ void k_lz_load(Dev D, int which) {
  const ProbDesc& p = D.P[blockIdx.y];
  const ProbState& st = D.st[blockIdx.y];
  if (st.done) return;
  const float2* src = lz_col(D, which ? BUF_U : BUF_V, p, st.lk);
  float2* dst = lz_col(D, BUF_B1, p, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// B2[:, 0] -= beta_k u_{k-1} (which = 0, k > 0) or alpha_k v_k (which = 1): the three-term part.
__global__ void k_lz_axpy(Dev D, int which) {
  const ProbDesc& p = D.P[blockIdx.y];
  const ProbState& st = D.st[blockIdx.y];
  if (st.done) return;
  if (which == 0 && st.lk == 0) return;
  const float coef = (float)(which ? st.lalpha : st.lbeta);
  const float2* x = which ? lz_col(D, BUF_V, p, st.lk) : lz_col(D, BUF_U, p, st.lk - 1);
  float2* r = lz_col(D, BUF_B2, p, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += gridDim.x * blockDim.x)
    r[i] = make_float2(r[i].x - coef * x[i].x, r[i].y - coef * x[i].y);
}

// norm of B2[:, 0]; accept it as u_k (which = 0, alpha) or v_{k+1} (which = 1, beta), or stop.
__global__ void k_lz_accept(Dev D, int which, double tol_rel, int cap) {
  __shared__ float sh[32];
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (st.done) return;
  const float2* r = lz_col(D, BUF_B2, p, 0);
  float acc = 0.f;
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) acc += r[i].x * r[i].x + r[i].y * r[i].y;
  const double nrm = sqrt((double)block_sum_f(acc, sh));
  const double tol = tol_rel * sqrt(fmax(st.normT2, 0.0));
  const bool stop = !(nrm > tol) || !isfinite(nrm);
  const int k = st.lk;
  const bool room = which == 0 || k + 2 <= min(cap, p.r0);   // v_{k+1} goes to column k + 1 < r0
  if (!stop && room) {
    float2* dst = which ? lz_col(D, BUF_V, p, k + 1) : lz_col(D, BUF_U, p, k);
    const float inv = (float)(1.0 / nrm);
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) dst[i] = make_float2(r[i].x * inv, r[i].y * inv);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (which == 0) {
      if (stop) {
        st.lstop = 1;                               // alpha: v_0 .. v_k stay, u_k does not
        st.done = 1;
      } else {
        st.lalpha = nrm;
      }
    } else {
      st.lk = k + 1;                                // u_k accepted
      if (stop || !room) {
        st.lstop = stop ? 2 : 3;                    // beta, or the block is full: v_0 .. v_k
        st.done = 1;
      } else {
        st.lbeta = nrm;
      }
    }
  }
}

// After the iteration every right vector computed starts the power iteration: v_0 .. v_k (k
// accepted u) when alpha stopped it, v_0 .. v_{k-1} otherwise.  After an alpha stop with v_0
// outside the range of T^*, only the k + 1 vectors together contain that range (Section 2.1):
// T [v_0 .. v_k] has the singular values of T, while T [v_0 .. v_{k-1}] can be close to
// singular.  Every problem takes part again.
__global__ void k_lz_finish(Dev D) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= D.nprob) return;
  ProbState& s = D.st[pi];
  if (s.status == ST_ENAN) return;                  // non-finite input stays excluded
  s.wv = min(max(s.lk + (s.lstop == 1 ? 1 : 0), 1), D.P[pi].r0);
  s.wu = s.wv;
  s.rank_det = s.lk;
  s.done = 0;
}

__global__ void k_lz_all_done(Dev D, int* flag) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= D.nprob) return;
  if (!D.st[pi].done) atomicExch(flag, 0);
}

inline dim3 col_grid(const Dev& D) { return dim3(std::max(1, std::min((D.maxN + 255) / 256, 64)), D.nprob); }

}  // namespace

void launch_lz_start(const Dev& D, cudaStream_t s) {
  note_launch();
  k_lz_start<<<D.nprob, 256, 0, s>>>(D);
}
void launch_lz_load(const Dev& D, int which, cudaStream_t s) {
  note_launch();
  k_lz_load<<<col_grid(D), 256, 0, s>>>(D, which);
}
void launch_lz_axpy(const Dev& D, int which, cudaStream_t s) {
  note_launch();
  k_lz_axpy<<<col_grid(D), 256, 0, s>>>(D, which);
}
void launch_lz_accept(const Dev& D, int which, double tol_rel, int cap, cudaStream_t s) {
  note_launch();
  k_lz_accept<<<D.nprob, 256, 0, s>>>(D, which, tol_rel, cap);
}
void launch_lz_finish(const Dev& D, cudaStream_t s) {
  note_launch();
  k_lz_finish<<<(D.nprob + 127) / 128, 128, 0, s>>>(D);
}
void launch_lz_all_done(const Dev& D, int* flag, cudaStream_t s) {
  note_launch();
  k_lz_all_done<<<(D.nprob + 127) / 128, 128, 0, s>>>(D, flag);
}
