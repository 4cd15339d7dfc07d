// Toeplitz block products of the power iterations (Algorithm 3) and of the S_l
// generation (Eq. generateSl):
//     Y[k, j] = sum_{h in I_n} F(k - h) X[h, j],
// F = f for T (and, over the row box {0..n+1}^d, for every T_l at once) or
// F(x) = conj f(-x) for T^*.  The multilevel Toeplitz matrix is never formed:
// each tile is generated from the sample grid, whose linear index of k - h is
// gk(k) - gh(h) with gk(k) = sum_l (k_l + n) G^(d-1-l), gh(h) = sum_l h_l G^(d-1-l).
//
// This file holds the FP32 CUDA-core kernel (PRONY_FP32).  Work is a list of
// jobs (problem, 64-row tile, K split) over all problems of a batch, the K splits of a tile
// consecutive.  With a K split every CTA of a tile stores its partial sums in a workspace slot
// and the last to arrive (a per-tile counter) adds them in the order of their K ranges, so the
// result does not depend on the order in which the CTAs finish.
#include "common.cuh"
#include <algorithm>
#include <climits>

namespace {

constexpr int TBM = 64;    // output rows per block

__device__ inline float2* tbuf(const Dev& D, int buf, const ProbDesc& p, int& ld) {
  switch (buf) {
    case BUF_V: ld = p.N; return D.V + p.xoff;
    case BUF_U: ld = p.N; return D.U + p.xoff;
    case BUF_B1: ld = p.N; return D.B1 + p.xoff;
    case BUF_B2: ld = p.N; return D.B2 + p.xoff;
    default: ld = p.Next; return D.Y + p.yoff;
  }
}

__device__ inline int twidth(const ProbState& s, const ProbDesc& p, int sel) { return sel_width(s, p, sel); }

template <int TN, int TBK>
__global__ void __launch_bounds__(256) k_toeplitz_simt(Dev D, const ToeplitzJob* jobs, int adjoint, int xbuf,
                                                       int wsel, int ybuf, int y_ext, float2* part, int* cnt,
                                                       int maxw, long long part_jobs) {
  constexpr int NCOL = 16 * TN;
  __shared__ int gk[TBM];
  __shared__ int gh[TBK];
  __shared__ float2 As[TBK][TBM];
  __shared__ float2 Xs[TBK][NCOL];
  const ToeplitzJob job = jobs[blockIdx.x];
  const ProbDesc& p = D.P[job.prob];
  const ProbState& st = D.st[job.prob];
  if (st.done) return;
  const int w = twidth(st, p, wsel);
  if (w <= 0) return;
  const int L = y_ext ? p.n + 2 : p.n + 1;
  const int rows_total = y_ext ? p.Next : p.N;
  const int row0 = job.mt * TBM;
  if (row0 >= rows_total) return;
  const int chunk = ((p.N + job.nks - 1) / job.nks + TBK - 1) / TBK * TBK;
  const int kb = job.ks * chunk, ke = min(p.N, kb + chunk);
  if (kb >= ke && job.nks == 1) return;       // (an empty K range of a split still reports zeros)
  const float2* F = (adjoint ? D.gH : D.gF) + p.grid;
  int ldx, ldy;
  const float2* X = tbuf(D, xbuf, p, ldx);
  float2* Y = tbuf(D, ybuf, p, ldy);

  for (int i = threadIdx.x; i < TBM; i += blockDim.x) {
    int row = row0 + i, g = -1;
    if (row < rows_total) {
      int rem = row, mul = 1;
      g = 0;
      for (int l = p.d - 1; l >= 0; --l) {
        g += (rem % L + p.n) * mul;
        rem /= L;
        mul *= p.G;
      }
    }
    gk[i] = g;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);

  for (int h0 = kb; h0 < ke; h0 += TBK) {
    __syncthreads();
    if (threadIdx.x < TBK) {
      int h = h0 + (int)threadIdx.x, g = 0;
      if (h < ke) {
        int rem = h, mul = 1;
        for (int l = p.d - 1; l >= 0; --l) {
          g += (rem % (p.n + 1)) * mul;
          rem /= (p.n + 1);
          mul *= p.G;
        }
      } else {
        g = INT_MIN;
      }
      gh[threadIdx.x] = g;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TBK * TBM; idx += blockDim.x) {
      int kk = idx / TBM, i = idx % TBM;
      int g1 = gk[i], g2 = gh[kk];
      As[kk][i] = (g1 >= 0 && g2 != INT_MIN) ? F[g1 - g2] : make_float2(0.f, 0.f);
    }
    for (int idx = threadIdx.x; idx < TBK * NCOL; idx += blockDim.x) {
      int kk = idx % TBK, c = idx / TBK;
      int h = h0 + kk;
      Xs[kk][c] = (c < w && h < ke) ? X[(long long)c * ldx + h] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TBK; ++kk) {
      float2 a[4], x[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) x[j] = Xs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fmaf(a[i].x, x[j].x, fmaf(-a[i].y, x[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, x[j].y, fmaf(a[i].y, x[j].x, acc[i][j].y));
        }
    }
  }
  if (job.nks == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int row = row0 + ty * 4 + i;
      if (row >= rows_total) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int c = tx + 16 * j;
        if (c < w) Y[(long long)c * ldy + row] = acc[i][j];
      }
    }
    return;
  }
  // split K: partial tile into this job's slot (column c, row i at c * TBM + i), then one arrival
  __shared__ int s_last;
  const size_t slot = (size_t)maxw * TBM;
  float2* mine = part + (size_t)blockIdx.x * slot;
  const bool mine_ok = ws_ok(D, (long long)blockIdx.x - job.ks + job.nks <= part_jobs && w <= maxw, 22);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = tx + 16 * j;
      if (c < w && mine_ok) mine[(size_t)c * TBM + ty * 4 + i] = acc[i][j];
    }
  __threadfence();
  __syncthreads();
  const int first_job = blockIdx.x - job.ks;
  if (threadIdx.x == 0) s_last = mine_ok && atomicAdd(&cnt[first_job], 1) == job.nks - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const float2* base = part + (size_t)first_job * slot;
  for (int idx = threadIdx.x; idx < w * TBM; idx += blockDim.x) {
    const int c = idx / TBM, i = idx % TBM, row = row0 + i;
    float2 v = __ldcg(base + idx);
    for (int k = 1; k < job.nks; ++k) {
      const float2 u = __ldcg(base + (size_t)k * slot + idx);
      v.x += u.x;
      v.y += u.y;
    }
    if (row < rows_total) Y[(long long)c * ldy + row] = v;
  }
  if (threadIdx.x == 0) cnt[first_job] = 0;   // ready for the next launch
}

template <int TN>
void run_simt(const Dev& D, const ToeplitzJob* jobs, int njobs, int adjoint, int xbuf, int wsel, int ybuf, int y_ext,
              float2* part, int* cnt, int maxw, long long part_jobs, cudaStream_t s) {
  constexpr int KB = TN > 5 ? 16 : 32;   // keep the static tiles under 48 KB
  note_launch();
  k_toeplitz_simt<TN, KB><<<njobs, 256, 0, s>>>(D, jobs, adjoint, xbuf, wsel, ybuf, y_ext, part, cnt, maxw,
                                                  part_jobs);
}

}  // namespace

size_t simt_part_elems(int maxw) { return (size_t)maxw * TBM; }

void launch_toeplitz(const Dev& D, const ToeplitzJob* jobs, int njobs, int adjoint, int xbuf, int wsel, int ybuf,
                     int y_ext, int maxw, float2* part, int* cnt, long long part_jobs, cudaStream_t s) {
  int tn = (maxw + 15) / 16;
  if (tn <= 1) run_simt<1>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, part, cnt, maxw, part_jobs, s);
  else if (tn <= 2) run_simt<2>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, part, cnt, maxw, part_jobs, s);
  else if (tn <= 3) run_simt<3>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, part, cnt, maxw, part_jobs, s);
  else if (tn <= 5) run_simt<5>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, part, cnt, maxw, part_jobs, s);
  else run_simt<8>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, part, cnt, maxw, part_jobs, s);
}
