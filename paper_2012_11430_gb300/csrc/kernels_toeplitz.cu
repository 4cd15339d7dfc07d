// Toeplitz block products of the power iterations (Algorithm 3) and of the S_l
// generation (Eq. generateSl):
//     Y[k, j] = sum_{h in I_n} F(k - h) X[h, j],
// F = f for T (and, over the row box {0..n+1}^d, for every T_l at once) or
// F(x) = conj f(-x) for T^*.  The multilevel Toeplitz matrix is never formed:
// each tile is generated from the sample grid, whose linear index of k - h is
// gk(k) - gh(h) with gk(k) = sum_l (k_l + n) G^(d-1-l), gh(h) = sum_l h_l G^(d-1-l).
//
// This file holds the FP32 CUDA-core kernel (PRONY_FP32).  Work is a list of
// jobs (problem, 64-row tile, K split) over all problems of a batch; partial sums
// of the K splits meet in Y with atomics (Y zeroed per live problem first).
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

__global__ void k_zero_buf(Dev D, int buf, int wsel, int y_ext) {
  const ProbDesc& p = D.P[blockIdx.y];
  const ProbState& s = D.st[blockIdx.y];
  if (s.done) return;
  int ld;
  float2* Yb = tbuf(D, buf, p, ld);
  const int w = twidth(s, p, wsel);
  const long long rows = y_ext ? p.Next : p.N;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < rows * w;
       q += (long long)gridDim.x * blockDim.x) {
    int c = (int)(q / rows);
    long long r = q % rows;
    Yb[(long long)c * ld + r] = make_float2(0.f, 0.f);
  }
}

template <int TN, int TBK>
__global__ void __launch_bounds__(256) k_toeplitz_simt(Dev D, const ToeplitzJob* jobs, int adjoint, int xbuf,
                                                       int wsel, int ybuf, int y_ext) {
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
  if (kb >= ke) return;
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
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int row = row0 + ty * 4 + i;
    if (row >= rows_total) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int c = tx + 16 * j;
      if (c < w) {
        float2* yp = &Y[(long long)c * ldy + row];
        if (job.nks == 1) {
          *yp = acc[i][j];
        } else {
          atomicAdd(&yp->x, acc[i][j].x);
          atomicAdd(&yp->y, acc[i][j].y);
        }
      }
    }
  }
}

template <int TN>
void run_simt(const Dev& D, const ToeplitzJob* jobs, int njobs, int adjoint, int xbuf, int wsel, int ybuf, int y_ext,
              cudaStream_t s) {
  constexpr int KB = TN > 5 ? 16 : 32;   // keep the static tiles under 48 KB
  note_launch();
  k_toeplitz_simt<TN, KB><<<njobs, 256, 0, s>>>(D, jobs, adjoint, xbuf, wsel, ybuf, y_ext);
}

}  // namespace

void launch_zero_buf(const Dev& D, int buf, int wsel, int y_ext, cudaStream_t s) {
  dim3 g(64, D.nprob);
  note_launch();
  k_zero_buf<<<g, 256, 0, s>>>(D, buf, wsel, y_ext);
}

void launch_toeplitz(const Dev& D, const ToeplitzJob* jobs, int njobs, int nks, int adjoint, int xbuf, int wsel,
                     int ybuf, int y_ext, int maxw, int precision, cudaStream_t s) {
  (void)precision;
  if (nks > 1) launch_zero_buf(D, ybuf, wsel, y_ext, s);
  int tn = (maxw + 15) / 16;
  if (tn <= 1) run_simt<1>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, s);
  else if (tn <= 2) run_simt<2>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, s);
  else if (tn <= 3) run_simt<3>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, s);
  else if (tn <= 5) run_simt<5>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, s);
  else run_simt<8>(D, jobs, njobs, adjoint, xbuf, wsel, ybuf, y_ext, s);
}
