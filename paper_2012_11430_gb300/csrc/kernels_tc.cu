// Tensor-core (tcgen05) Toeplitz block products for sm_103a.
//
// Y[k, j] = sum_{h in I_n} F(k - h) X[h, j]  (F = f for T, conj f(-x) for T^*), as the real GEMM
//   Y' (rows x 2w) = A' (rows x 2N) * B' (2N x 2w),
// A' row k, K-chunk c (32 input points h = 32c .. 32c+31) = [Re F(k-h) | Im F(k-h)] (64 real K),
// B' column 2j (Re Y_j) = [Re X_j ; -Im X_j], column 2j+1 (Im Y_j) = [Im X_j ; Re X_j].
// FP32 operands are split into BF16 planes (x = x0 + x1 [+ x2]); the products x_a y_b with
// a + b <= NPL - 1 are accumulated in FP32 in tensor memory (3 products for two planes,
// 6 for three planes, which represent FP32 inputs exactly).
//
// One CTA = 128 output rows x all 2w columns x a range of K chunks.  Warp roles:
//   warp 0  TMA: the sample-grid window (one bulk copy) and the B' tiles (2-D tiled, 128B swizzle)
//   warp 1  MMA issue (one thread), tcgen05.commit to the stage barriers
//   warps 2-5  generate the Toeplitz A' tile of each chunk from the window in shared memory and
//           write its BF16 planes straight into tensor memory (tcgen05.st); then the epilogue
// The Toeplitz matrix is never formed in HBM: each A' element is F at grid index gk(k) - gh(h).
#include "common.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstring>

namespace {

constexpr int TC_BM = 128;
constexpr uint32_t TC_SPIN = 1u << 24;      // bounded mbarrier polls (~seconds)
constexpr int TC_A_COL0 = 256;              // TMEM: D in columns [0, 256), A stages from 256

__device__ inline int tc_width(const ProbState& s, const ProbDesc& p, int sel) {
  switch (sel) {
    case W_R0: return p.r0;
    case W_U: return s.wu;
    case W_V: return s.wv;
    case W_M: return p.m;
    case W_IN: return s.w_in;
    default: return s.w_out;
  }
}

__device__ inline float2* tc_buf(const Dev& D, int buf, const ProbDesc& p, int& ld) {
  switch (buf) {
    case BUF_V: ld = p.N; return D.V + p.xoff;
    case BUF_U: ld = p.N; return D.U + p.xoff;
    case BUF_B1: ld = p.N; return D.B1 + p.xoff;
    case BUF_B2: ld = p.N; return D.B2 + p.xoff;
    default: ld = p.Next; return D.Y + p.yoff;
  }
}

// grid linear index of a point of the box {0..L-1}^d shifted by +n in every coordinate
__device__ inline int grid_of_row(int row, int L, const ProbDesc& p) {
  int g = 0, mul = 1, rem = row;
  for (int l = p.d - 1; l >= 0; --l) {
    g += (rem % L + p.n) * mul;
    rem /= L;
    mul *= p.G;
  }
  return g;
}
__device__ inline int grid_of_h(int h, const ProbDesc& p) {
  int g = 0, mul = 1, rem = h;
  for (int l = p.d - 1; l >= 0; --l) {
    g += (rem % (p.n + 1)) * mul;
    rem /= (p.n + 1);
    mul *= p.G;
  }
  return g;
}

// Split an FP32 pair into BF16x2 planes (exact for three planes).
template <int NPL>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t* w) {
  uint32_t h = pack_bf16x2(a, b);
  w[0] = h;
  float ra = a - bf16lo_to_f32(h), rb = b - bf16hi_to_f32(h);
  uint32_t m = pack_bf16x2(ra, rb);
  w[1] = m;
  if (NPL == 3) {
    ra -= bf16lo_to_f32(m);
    rb -= bf16hi_to_f32(m);
    w[2] = pack_bf16x2(ra, rb);
  }
}

// X (N x w complex64, column-major) -> B' planes: row 2j / 2j+1 of plane p, K index 64c + q.
__global__ void k_xb_prep(Dev D, int xbuf, int wsel, uint16_t* xb, int npl, int ntbox, int kpitch) {
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  const ProbState& s = D.st[pi];
  if (s.done) return;
  const int w = tc_width(s, p, wsel);
  const int nt = ((2 * w + 15) / 16) * 16;
  const int nc = (p.N + 31) / 32;
  int ldx;
  const float2* X = tc_buf(D, xbuf, p, ldx);
  uint16_t* out = xb + (size_t)pi * npl * ntbox * kpitch;
  const long long total = (long long)nt * nc * 32;        // (row, chunk, point-in-chunk)
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    int jj = (int)(q % 32);
    long long t = q / 32;
    int c = (int)(t % nc);
    int row = (int)(t / nc);
    int h = 32 * c + jj;
    int j = row >> 1;
    float2 x = (h < p.N && j < w) ? X[(long long)j * ldx + h] : make_float2(0.f, 0.f);
    float vr, vi;                          // value in the Re-F block (q < 32) and the Im-F block (q >= 32)
    if ((row & 1) == 0) { vr = x.x; vi = -x.y; }
    else { vr = x.y; vi = x.x; }
    // split both values; planes stored at [plane][row][kpitch]
    uint32_t wr[3];
    if (npl == 3) split_pair<3>(vr, vi, wr);
    else split_pair<2>(vr, vi, wr);
    for (int pl = 0; pl < npl; ++pl) {
      uint16_t* dst = out + ((size_t)pl * ntbox + row) * kpitch + 64 * c;
      dst[jj] = (uint16_t)(wr[pl] & 0xFFFF);
      dst[32 + jj] = (uint16_t)(wr[pl] >> 16);
    }
  }
}

struct TcParams {
  int adjoint, xbuf_unused, wsel, ybuf, y_ext;
  int ntbox, kpitch, win_cap;     // TMA box rows, K pitch of B', window capacity (float2 entries)
  int stages;
};

template <int NPL>
__global__ void __launch_bounds__(192, 1) k_toeplitz_tc(Dev D, const ToeplitzJob* jobs, TcParams P,
                                                        const __grid_constant__ CUtensorMap bmap, int* err) {
  constexpr int NPROD = NPL == 3 ? 6 : 3;
  constexpr int PA[6] = {0, 0, 1, 0, 1, 2};
  constexpr int PB[6] = {0, 1, 0, 2, 1, 0};
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_win, bar_d;
  __shared__ uint64_t bar_bfull[4], bar_afull[4], bar_empty[4];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;

  const ToeplitzJob job = jobs[blockIdx.x];
  const ProbDesc& p = D.P[job.prob];
  const ProbState& st = D.st[job.prob];
  if (st.done) return;
  const int w = tc_width(st, p, P.wsel);
  if (w <= 0) return;
  const int L = P.y_ext ? p.n + 2 : p.n + 1;
  const int rows_total = P.y_ext ? p.Next : p.N;
  const int row0 = job.mt * TC_BM;
  if (row0 >= rows_total) return;
  const int nc = (p.N + 31) / 32;
  const int cper = (nc + job.nks - 1) / job.nks;
  const int c_begin = job.ks * cper, c_end = min(nc, c_begin + cper);
  if (c_begin >= c_end) return;
  const int nchunks = c_end - c_begin;
  const int NT = ((2 * w + 15) / 16) * 16;
  const int S = P.stages;

  // window of grid indices needed by this CTA: [gk(first row) - gh(last h), gk(last row) - gh(first h)]
  const int last_row = min(rows_total, row0 + TC_BM) - 1;
  const int h_first = 32 * c_begin, h_last = min(p.N, 32 * c_end) - 1;
  int wlo = grid_of_row(row0, L, p) - grid_of_h(h_last, p);
  int whi = grid_of_row(last_row, L, p) - grid_of_h(h_first, p);
  wlo &= ~1;                                  // 16-byte aligned start (float2 pairs)
  int wlen = whi - wlo + 1;
  wlen = (wlen + 1) & ~1;
  if (wlen > P.win_cap) {                     // host sizing guarantees this does not happen
    if (threadIdx.x == 0) atomicExch(err, 3);
    return;
  }
  const float2* F = (P.adjoint ? D.gH : D.gF) + p.grid;

  // shared memory: B stages (1024-aligned), then the window
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const uint32_t stage_bytes = (uint32_t)NPL * P.ntbox * 128u;
  unsigned char* Bs = sm;
  float2* win = (float2*)(sm + (size_t)S * stage_bytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    tmem_alloc(&s_tmem, 512);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    mbar_init(&bar_win, 1);
    mbar_init(&bar_d, 1);
    for (int i = 0; i < S; ++i) {
      mbar_init(&bar_bfull[i], 1);
      mbar_init(&bar_afull[i], 4);
      mbar_init(&bar_empty[i], 1);
    }
    s_err = 0;
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = s_tmem;

  if (warp == 0) {
    // ------------------------------------------------------------- TMA producer
    if (lane == 0) {
      mbar_arrive_expect_tx(&bar_win, (uint32_t)wlen * 8u);
      tma_load_1d(win, F + wlo, (uint32_t)wlen * 8u, &bar_win);
      const int yrow0 = job.prob * NPL * P.ntbox;
      int issued = 0;
      for (int it = 0; it < nchunks; ++it) {
        const int s = it % S, u = it / S;
        if (it >= S && !mbar_wait(&bar_empty[s], (u - 1) & 1, TC_SPIN)) { s_err = 1; break; }
        mbar_arrive_expect_tx(&bar_bfull[s], stage_bytes);
        for (int pl = 0; pl < NPL; ++pl)
          tma_load_2d(Bs + (size_t)s * stage_bytes + (size_t)pl * P.ntbox * 128, &bmap, 64 * (c_begin + it),
                      yrow0 + pl * P.ntbox, &bar_bfull[s]);
        ++issued;
      }
      // in-flight copies end before the CTA exits
      if (issued > 0) {
        const int last = issued - 1;
        mbar_wait(&bar_bfull[last % S], (last / S) & 1, TC_SPIN);
      }
      mbar_wait(&bar_win, 0, TC_SPIN);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(TC_BM, NT);
      for (int it = 0; it < nchunks; ++it) {
        const int s = it % S, u = it / S;
        if (!mbar_wait(&bar_afull[s], u & 1, TC_SPIN) || !mbar_wait(&bar_bfull[s], u & 1, TC_SPIN)) {
          s_err = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = tb + TC_A_COL0 + (uint32_t)s * NPL * 32;
        const uint32_t bsm = smem_u32(Bs + (size_t)s * stage_bytes);
#pragma unroll
        for (int pr = 0; pr < NPROD; ++pr) {
          const uint32_t a_pl = a0 + PA[pr] * 32;
          const uint64_t bd = sdesc_sw128(bsm + PB[pr] * P.ntbox * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_ts_f16(tb, a_pl + 8 * kk, bd + 2 * kk, idesc, (it > 0 || pr > 0 || kk > 0) ? 1u : 0u);
        }
        tc_commit(&bar_empty[s]);
      }
      tc_commit(&bar_d);      // arrives when every MMA issued above has completed
    }
  } else {
    // ------------------------------------------------------------- A producers + epilogue
    const int q = warp & 3;                     // TMEM lane quadrant of this warp
    const int i = 32 * q + lane;                // row within the tile
    const int row = row0 + i;
    const bool vrow = row < rows_total;
    const int gk = vrow ? grid_of_row(row, L, p) - wlo : 0;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_win, 0, TC_SPIN));
    if (!ok) s_err = 1;
    for (int it = 0; ok && it < nchunks; ++it) {
      const int s = it % S, u = it / S;
      if (it >= S && !__all_sync(0xffffffffu, mbar_wait(&bar_empty[s], (u - 1) & 1, TC_SPIN))) {
        s_err = 1;
        break;
      }
      const int h = 32 * (c_begin + it) + lane;
      const int ghl = h < p.N ? grid_of_h(h, p) : INT_MIN;
      float re[32], im[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int g = __shfl_sync(0xffffffffu, ghl, j);
        float2 v = make_float2(0.f, 0.f);
        if (vrow && g != INT_MIN) v = win[gk - g];
        re[j] = v.x;
        im[j] = v.y;
      }
      const uint32_t a0 = tb + lane_off + TC_A_COL0 + (uint32_t)s * NPL * 32;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const float* src = half ? im : re;
        uint32_t wp[NPL][16];
#pragma unroll
        for (int jp = 0; jp < 16; ++jp) {
          uint32_t t3[3];
          split_pair<NPL>(src[2 * jp], src[2 * jp + 1], t3);
#pragma unroll
          for (int pl = 0; pl < NPL; ++pl) wp[pl][jp] = t3[pl];
        }
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) tmem_st_x16(a0 + pl * 32 + half * 16, wp[pl]);
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_afull[s]);
    }
    // epilogue: D (TMEM) -> Y
    if (__all_sync(0xffffffffu, mbar_wait(&bar_d, 0, TC_SPIN)) && !s_err) {
      tc_fence_after();
      int ldy;
      float2* Y = tc_buf(D, P.ybuf, p, ldy);
      for (int c0 = 0; c0 < NT; c0 += 16) {
        uint32_t v[16];
        tmem_ld_x16(tb + lane_off + c0, v);
        tmem_ld_wait();
        if (vrow) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = c0 / 2 + e;
            if (j < w) {
              float2 val = make_float2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]));
              float2* yp = &Y[(long long)j * ldy + row];
              if (job.nks == 1) *yp = val;
              else atomicAdd(yp, val);
            }
          }
        }
      }
    } else {
      s_err = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_err && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 0) {
    tc_fence_after();
    // on an error path, let the MMAs already issued finish before the columns are released
    if (s_err) mbar_wait(&bar_d, 0, TC_SPIN);
    tmem_dealloc(tb, 512);
  }
}

}  // namespace

// ----------------------------------------------------------------------------- host side
// Tensor map over the B' buffer: 2-D, inner dimension K (kpitch BF16), outer rows, 128B swizzle.
// The driver's tensor-map encoder, looked up through the runtime (the library does not link
// libcuda, so it also loads on machines without a GPU driver).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

int encode_xb_map(CUtensorMap* map, void* xb, int kpitch, long long rows, int ntbox) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return -1;
  cuuint64_t dims[2] = {(cuuint64_t)kpitch, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpitch * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)ntbox};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xb, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

size_t tc_smem_bytes(int npl, int ntbox, int stages, int win_cap) {
  return 1024 + (size_t)stages * npl * ntbox * 128 + (size_t)win_cap * 8;
}

void launch_xb_prep(const Dev& D, int xbuf, int wsel, void* xb, int npl, int ntbox, int kpitch, cudaStream_t s) {
  note_launch();
  dim3 g(std::max(1, std::min(((D.maxN + 31) / 32) * 4, 1024)), D.nprob);
  k_xb_prep<<<g, 256, 0, s>>>(D, xbuf, wsel, (uint16_t*)xb, npl, ntbox, kpitch);
}

void launch_toeplitz_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int nks, int adjoint, int wsel, int ybuf,
                        int y_ext, int npl, int ntbox, int kpitch, int win_cap, int stages, const CUtensorMap& map,
                        int* err, cudaStream_t s) {
  if (nks > 1) launch_zero_buf(D, ybuf, wsel, y_ext, s);
  TcParams P{adjoint, 0, wsel, ybuf, y_ext, ntbox, kpitch, win_cap, stages};
  size_t sm = tc_smem_bytes(npl, ntbox, stages, win_cap);
  note_launch();
  // the attribute must cover this launch's dynamic shared memory (static + dynamic <= 227 KB)
  if (npl == 3) {
    static size_t set3 = 0;
    if (sm > set3) {
      cudaFuncSetAttribute(k_toeplitz_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set3 = sm;
    }
    k_toeplitz_tc<3><<<njobs, 192, sm, s>>>(D, jobs, P, map, err);
  } else {
    static size_t set2 = 0;
    if (sm > set2) {
      cudaFuncSetAttribute(k_toeplitz_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set2 = sm;
    }
    k_toeplitz_tc<2><<<njobs, 192, sm, s>>>(D, jobs, P, map, err);
  }
}
