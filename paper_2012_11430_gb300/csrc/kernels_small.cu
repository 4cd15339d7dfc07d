// Small per-problem kernels (one thread block per problem of a batch).
//
//  k_chol     FP32 Cholesky of the Gram X^* X with diagonal pivoting: the R factor of a
//             column-pivoted QR (Algorithm 3, lines with QR / QR with column pivoting),
//             the rank criterion ||R(i:r0,i:r0)||_F <= tol ||R||_F (Section 2.2) read off the
//             trailing Schur-complement trace, and the map X -> X P R^{-1}.
//  k_solve_c  FP64 Vandermonde Gram conj(A) A^T (product of Dirichlet kernels) and Cholesky
//             solve of the normal equations of Eq. ls_probl; results sorted by t.
// All loops are bounded; a cap that is hit sets PRONY_ENOCONV in the problem's state.
#include "common.cuh"
#include <algorithm>


namespace {

__device__ inline int swidth(const ProbState& s, const ProbDesc& p, int sel) { return sel_width(s, p, sel); }
__device__ inline void set_width(ProbState& s, int sel, int w) {
  if (sel == W_U) s.wu = w;
  else if (sel == W_V) s.wv = w;
}
__device__ inline void set_status(ProbState& s, int st) {
  if (s.status == ST_OK) s.status = st;
}

// ----------------------------------------------------------------------------- pivoted Cholesky (FP32)
// Step i: warp 0 finds the pivot (largest remaining diagonal entry, lowest index on ties) and the
// trailing trace and decides whether to stop; rows and columns i, pv are swapped; the scaled
// column l = A[:, i] / sqrt(A[i][i]) goes to shared memory and the trailing block takes the rank-1
// update A[j][k] -= l_j conj(l_k).  R^{-1} (R = L^H) is formed by one warp per column with the
// partial sums of the back substitution spread over the lanes.
__global__ void __launch_bounds__(256) k_chol(Dev D, int wsel, int target, int mode_in, double tol, int rank_mode) {
  extern __shared__ float2 A[];                 // [w][LDR]
  __shared__ int perm[PRONY_RMAX];
  __shared__ float2 lcol[PRONY_RMAX];
  __shared__ int s_piv, s_stop, s_rho, s_rank;
  __shared__ float s_trace0, s_maxd0;
  const ProbDesc& p = D.P[blockIdx.x];
  ProbState& st = D.st[blockIdx.x];
  if (st.done) return;
  // QR_AUTO: the rank step (column pivoting and rank test, Algorithm 3) on a problem's first
  // power iteration, plain CholeskyQR afterwards
  const int mode = mode_in == QR_AUTO ? (st.iter == 0 ? QR_RANK : QR_PLAIN) : mode_in;
  const int w = swidth(st, p, wsel);
  const int LR = D.L.LDR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double2* G = (const double2*)(D.small + p.soff + D.L.gram);
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    int i = idx / w, j = idx % w;
    double2 g = G[i * LR + j];
    A[i * LR + j] = make_float2((float)g.x, (float)g.y);
  }
  for (int i = threadIdx.x; i < w; i += blockDim.x) perm[i] = i;
  __syncthreads();
  if (warp == 0) {
    float tr = 0.f, mx = 0.f;
    bool finite = true;
    for (int i = lane; i < w; i += 32) {
      const float dd = A[i * LR + i].x;
      finite = finite && isfinite(dd);
      tr += fmaxf(dd, 0.f);
      mx = fmaxf(mx, dd);
    }
    for (int o = 16; o > 0; o >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      s_trace0 = tr;
      s_maxd0 = mx;
      s_rho = w;
      s_rank = -1;
      s_stop = finite && isfinite(tr) ? 0 : 2;
      if (s_stop) {                     // non-finite block: the problem stops with ENAN
        st.status = ST_ENAN;
        st.done = 1;
        st.w_in = w;
        st.w_out = 0;
        set_width(st, target, 0);
      }
    }
  }
  __syncthreads();
  if (s_stop) return;
  const float tol2 = (float)(tol * tol);
  int limit = w;  // columns that may be accepted (never more than m after the rank step)
  if (mode == QR_RANK) limit = min(w, p.m);
  for (int i = 0; i < w; ++i) {
    if (warp == 0) {                    // pivot search and trailing trace (no search without pivoting)
      float best = -1.f, tr = 0.f;
      int bi = i;
      if (mode != QR_PLAIN) {
        for (int j = i + lane; j < w; j += 32) {
          const float dd = A[j * LR + j].x;
          tr += fmaxf(dd, 0.f);
          if (dd > best) {
            best = dd;
            bi = j;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          tr += __shfl_xor_sync(0xffffffffu, tr, o);
          const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
          const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
          if (b2 > best || (b2 == best && i2 < bi)) {
            best = b2;
            bi = i2;
          }
        }
      }
      if (lane == 0) {
        const int pv = (mode == QR_PLAIN) ? i : bi;
        const float dp = A[pv * LR + pv].x;
        if (mode == QR_RANK && s_rank < 0 && tr <= tol2 * s_trace0) s_rank = i;
        bool stop = false;
        if (!(dp > 1e-30f * s_maxd0) || !(dp > 0.f)) stop = true;                  // exhausted / not PD
        if (mode == QR_DROP && dp <= tol2 * s_maxd0) stop = true;
        if (i >= limit && (mode != QR_RANK || s_rank >= 0)) stop = true;
        if (mode == QR_RANK && rank_mode == 1 && s_rank >= 0) stop = true;
        if (stop) {
          s_stop = 1;
          s_rho = min(i, limit);
        }
        s_piv = pv;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int pv = s_piv;
    if (pv != i) {
      for (int j = threadIdx.x; j < w; j += blockDim.x) {  // swap rows i, pv
        const float2 t = A[i * LR + j];
        A[i * LR + j] = A[pv * LR + j];
        A[pv * LR + j] = t;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < w; j += blockDim.x) {  // swap cols i, pv
        const float2 t = A[j * LR + i];
        A[j * LR + i] = A[j * LR + pv];
        A[j * LR + pv] = t;
      }
      if (threadIdx.x == 0) {
        const int t = perm[i];
        perm[i] = perm[pv];
        perm[pv] = t;
      }
      __syncthreads();
    }
    const float inv = rsqrtf(A[i * LR + i].x);
    for (int j = i + threadIdx.x; j < w; j += blockDim.x) {
      const float2 v = A[j * LR + i];
      lcol[j] = make_float2(v.x * inv, v.y * inv);
    }
    __syncthreads();
    for (int j = i + threadIdx.x; j < w; j += blockDim.x) A[j * LR + i] = lcol[j];   // column i of L
    // rank-1 update of the trailing block: a warp per row (stepping by the warps), its lanes
    // over the columns (no index division)
    for (int j = i + 1 + warp; j < w; j += (int)(blockDim.x >> 5)) {
      const float2 lj = lcol[j];
#pragma unroll
      for (int q = 0; q < PRONY_RMAX / 32; ++q) {      // unrolled: the row's loads are issued together
        const int k = i + 1 + lane + 32 * q;
        if (k < w) {
          const float2 lk = lcol[k];
          float2 a = A[j * LR + k];
          a.x -= lj.x * lk.x + lj.y * lk.y;          // lj * conj(lk)
          a.y -= lj.y * lk.x - lj.x * lk.y;
          A[j * LR + k] = a;
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  const int rho = min(s_rho, limit);
  // R = L^H (rho x rho); M[perm[a]][b] = Rinv[a][b], column b by back substitution: x_b =
  // 1 / r_bb, then for k = b .. 0: x_k = s_k / r_kk and s_a -= R[a][k] x_k for a < k, the s_a
  // spread over the lanes of one warp (a = lane + 32 q).
  float2* M = (float2*)(D.small + p.soff + D.L.mapm);
  const int nwarp = blockDim.x >> 5;
  // reciprocals of the diagonal once (each column's substitution would otherwise divide at every
  // step of its dependent chain)
  __shared__ float rinv[PRONY_RMAX];
  for (int k = threadIdx.x; k < rho; k += blockDim.x) rinv[k] = 1.f / A[k * LR + k].x;
  __syncthreads();
  const int nq = (rho + 31) >> 5;
  for (int b = warp; b < rho; b += nwarp) {
    float2 sv[PRONY_RMAX / 32];
#pragma unroll
    for (int q = 0; q < PRONY_RMAX / 32; ++q) sv[q] = make_float2(lane + 32 * q == b ? 1.f : 0.f, 0.f);
    for (int k = b; k >= 0; --k) {
      const int ko = k & 31, kq = k >> 5;
      float2 mine = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < PRONY_RMAX / 32; ++q)
        if (q == kq) mine = sv[q];
      const float rk = rinv[k];
      const float2 xk = make_float2(__shfl_sync(0xffffffffu, mine.x, ko) * rk, __shfl_sync(0xffffffffu, mine.y, ko) * rk);
#pragma unroll
      for (int q = 0; q < PRONY_RMAX / 32; ++q) {
        if (q >= nq) break;
        const int a = lane + 32 * q;
        if (a == k) sv[q] = xk;
        else if (a < k) {
          const float2 l = A[k * LR + a];            // R[a][k] = conj(L[k][a])
          sv[q].x -= l.x * xk.x + l.y * xk.y;
          sv[q].y -= l.x * xk.y - l.y * xk.x;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PRONY_RMAX / 32; ++q) {
      const int a = lane + 32 * q;
      if (a < w) M[perm[a] * LR + b] = a <= b ? sv[q] : make_float2(0.f, 0.f);
    }
  }
  if (threadIdx.x == 0) {
    st.w_in = w;
    st.w_out = rho;
    set_width(st, target, rho);
    if (mode == QR_RANK) {
      st.rank_det = s_rank >= 0 ? s_rank : w;
      st.rank_used = rho;
      if (rho < p.m || st.rank_det < p.m) set_status(st, ST_ERANK);   // Section 2.2: rank below m
    }
    if (rho == 0) {
      set_status(st, ST_ERANK);
      st.done = 1;
    }
  }
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
  if (st.done || m <= 0 || m > p.m) return;
  double* t = (double*)(D.small + p.soff + D.L.t);
  double2* b = (double2*)(D.small + p.soff + D.L.rhs);
  double2* cout = (double2*)(D.small + p.soff + D.L.c);
  for (int q = threadIdx.x; q < m * d; q += blockDim.x) ts[(q / d) * PRONY_DMAX + q % d] = t[(q / d) * PRONY_DMAX + q % d];
  for (int i = threadIdx.x; i < m; i += blockDim.x) bb[i] = b[i];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // G[i][j] = prod_l sum_{x=0}^{n} exp(2 pi i (t_i(l) - t_j(l)) x), or with the raw eigenvalues
  // prod_l sum_x (conj(z_i(l)) z_j(l))^x (summed term by term: |q| need not be 1)
  const double2* zr = (const double2*)(D.small + p.soff + D.L.zraw);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    double2 g = make_double2(1.0, 0.0);
    if (D.vand) {
      for (int l = 0; l < d; ++l) {
        const double2 q = cmulc(zr[i * PRONY_DMAX + l], zr[j * PRONY_DMAX + l]);
        double2 sum = make_double2(1.0, 0.0), pw = make_double2(1.0, 0.0);
        for (int x = 1; x <= p.n; ++x) {
          pw = cmul(pw, q);
          sum = cadd(sum, pw);
        }
        g = cmul(g, sum);
      }
      G[i * LD + j] = g;
      continue;
    }
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
  if (threadIdx.x < 32) {
    // L y = b, then L^H c = y, column by column on one warp: lane l keeps the running residuals
    // r_j (j = l, l + 32); each step divides one residual by the diagonal and updates the
    // residuals of the rows that remain, so a step costs a few dependent FP64 operations instead
    // of a dot product of growing length
    const int lane = threadIdx.x;
    double2 r[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) r[q] = lane + 32 * q < m ? bb[lane + 32 * q] : make_double2(0.0, 0.0);
    for (int i = 0; i < m; ++i) {
      const int q = i >> 5;
      double2 ri = q ? r[1] : r[0];
      ri.x = __shfl_sync(0xffffffffu, ri.x, i & 31);
      ri.y = __shfl_sync(0xffffffffu, ri.y, i & 31);
      const double2 yi = cscale(ri, 1.0 / G[i * LD + i].x);
      if (lane == (i & 31)) cs_[i] = yi;
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int j = lane + 32 * qq;
        if (j > i && j < m) r[qq] = csub(r[qq], cmul(G[j * LD + i], yi));
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) r[q] = lane + 32 * q < m ? cs_[lane + 32 * q] : make_double2(0.0, 0.0);
    for (int i = m - 1; i >= 0; --i) {
      const int q = i >> 5;
      double2 ri = q ? r[1] : r[0];
      ri.x = __shfl_sync(0xffffffffu, ri.x, i & 31);
      ri.y = __shfl_sync(0xffffffffu, ri.y, i & 31);
      const double2 ci = cscale(ri, 1.0 / G[i * LD + i].x);
      if (lane == (i & 31)) cs_[i] = ci;
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int j = lane + 32 * qq;
        if (j < i) r[qq] = csub(r[qq], cmul(cconj(G[i * LD + j]), ci));
      }
    }
    if (lane == 0 && s_bad) set_status(st, ST_ERANK);
  }
  __syncthreads();
  // sort (t, c) lexicographically by t (and the raw eigenvalues with them)
  __shared__ double2 zs[PRONY_MMAX * PRONY_DMAX];
  double2* zw = (double2*)(D.small + p.soff + D.L.zraw);
  for (int q = threadIdx.x; q < m * d; q += blockDim.x) zs[(q / d) * PRONY_DMAX + q % d] = zw[(q / d) * PRONY_DMAX + q % d];
  __syncthreads();
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
    for (int l = 0; l < d; ++l) {
      t[r * PRONY_DMAX + l] = ts[j * PRONY_DMAX + l];
      zw[r * PRONY_DMAX + l] = zs[j * PRONY_DMAX + l];
    }
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
// A problem that failed (non-finite data, an empty U or V block, or a V block that never went
// through the rank step and is still wider than m) takes no part: rank_used = 0, so every
// finishing kernel skips it and its outputs are zero.
__global__ void k_reset_done(Dev D) {
  int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= D.nprob) return;
  ProbState& s = D.st[pi];
  const ProbDesc& p = D.P[pi];
  const bool failed = s.status == ST_ENAN || s.wv <= 0 || s.wu <= 0 || s.wv > p.m || s.wu > p.r0;
  if (failed) {
    if (s.status == ST_OK) set_status(s, ST_ERANK);
    s.rank_used = 0;
  }
  s.done = failed ? 1 : 0;
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

namespace {
// Condition of the device-side power loop: run the body again while some problem iterates and
// fewer than `cap` bodies ran (the cap bounds the loop whatever the flags say).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* all_done, int* count, int cap) {
  const int c = ++(*count);
  cudaGraphSetConditional(h, (*all_done == 0 && c < cap) ? 1u : 0u);
}
}  // namespace

void launch_loop_cond(cudaGraphConditionalHandle h, const int* all_done, int* count, int cap, cudaStream_t s) {
  note_launch();
  k_loop_cond<<<1, 1, 0, s>>>(h, all_done, count, cap);
}
