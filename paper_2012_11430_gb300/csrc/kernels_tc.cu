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
// B' depends on the problem and the K chunk only, so one small kernel (k_xb_prep) writes it once
// per product, already in the shared-memory image the MMA reads (planes stacked, rows of 128
// bytes, 128-byte swizzle), one contiguous tile per K chunk; a CTA moves a stage with one bulk
// copy.
//
// One CTA = 128 output rows x all 2w columns x a range of K chunks.  Warp roles:
//   warp 0      bulk copies: the CTA's window of the split-plane sample tables and every B' stage
//   warp 1      MMA issue (one thread): tcgen05.mma, A from tensor memory, B from shared memory
//   warps 2-9   A' producers: each chunk's Toeplitz tile is gathered from the window (its BF16
//               planes are split once per solve, k_split_tables, two input points per word) and
//               written straight into tensor memory (tcgen05.st); two warps per TMEM
//               lane quadrant, each taking half of the chunk's input points; then the epilogue
// The Toeplitz matrix is never formed in HBM: each A' element is F at grid index gk(k) - gh(h).
// A pipeline stage is one K chunk (its B' tile in shared memory and its A' tile in tensor
// memory); one full and one empty mbarrier per stage; every wait is bounded.
// Split K: the CTAs of one row tile (consecutive jobs) each store their FP32 partial tile in a
// workspace slot; the last of them to finish (a per-tile arrival counter) adds the partials in
// the order of their K ranges and writes Y, so results do not depend on which CTA ends first.
#include "common.cuh"
#include "tc_ptx.cuh"
#include "../../include/prony.h"

#include <algorithm>
#include <type_traits>
#include <climits>
#include <cstdlib>
#include <cstring>

namespace {

constexpr int TC_BM = 128;
constexpr uint32_t TC_SPIN = 1u << 24;      // bounded mbarrier polls (~seconds)
constexpr int TC_MAXSTAGE = 8;
constexpr int TC_APROD = 8;                 // A' warps (two per TMEM lane quadrant)
constexpr int TC_THREADS = 32 * (2 + TC_APROD);
constexpr int TC_MAXCH = 512;               // K chunks per CTA (host splits K to stay below)
enum TcMode { TC_PRODUCT = 0, TC_GRAM = 1, TC_APPLY = 2 };

__device__ inline int tc_width(const ProbState& s, const ProbDesc& p, int sel) { return sel_width(s, p, sel); }

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

// Split an FP32 value into TF32 hi + lo (round to nearest, ties away; both exactly TF32).
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32(float x, uint32_t* w) {
  const float hi = tf32_round(x);
  w[0] = __float_as_uint(hi);
  w[1] = __float_as_uint(tf32_round(x - hi));
}

// The three operand encodings.  Per 32-point K chunk (64 real K values) and plane:
//   BF16X3 / BF16X2  32 TMEM columns (two BF16 per column), 4 MMAs of K = 16, B rows of 128 bytes
//   TF32X3           64 TMEM columns (one TF32 per column), 8 MMAs of K = 8, B rows split into
//                    two 128-byte halves (K 0-31, 32-63), each a swizzle atom of its own
template <int KIND>
struct TcKind {
  static constexpr bool TF32 = KIND == PRONY_TF32X3;
  static constexpr int NPL = KIND == PRONY_BF16X3 ? 3 : 2;     // planes per operand
  static constexpr int NPROD = NPL == 3 ? 6 : 3;               // products a + b <= NPL - 1
  static constexpr int PCOLS = TF32 ? 64 : 32;                 // TMEM columns of a plane
  static constexpr int KSTEPS = TF32 ? 8 : 4;                  // MMAs per plane product and chunk
  static constexpr int KHALVES = TF32 ? 2 : 1;                 // 128-byte B row segments per chunk
  static constexpr int NTAB = 2 * NPL;                         // window tables (Re / Im x planes)
};

__device__ __forceinline__ void mma_ts(bool tf32, uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (tf32) mma_ts_tf32(d, a, b, idesc, acc);
  else mma_ts_f16(d, a, b, idesc, acc);
}

// X (N x w complex64, column-major) -> B' tiles.  B' row 2j / 2j+1 (output column), K index
// 64c + q (q < 32: Re-F block of input point 32c + q, q >= 32: Im-F block): row 2j holds
// (Re X_j, -Im X_j), row 2j+1 (Im X_j, Re X_j); rows from 2w up to NT are zero.  Chunk c of a
// problem is one contiguous tile in the shared-memory image of a B stage: KHALVES segments of
// NPL planes of NT rows of 128 bytes (BF16: 64 K per row; TF32: 32 K per row and segment), the
// 16-byte groups of row R swizzled by R mod 8 (the 128-byte swizzle of the MMA descriptor).
// One thread writes one 16-byte group of every plane.  Row h of X is row h of the buffer, or for
// the box buffer Y the row of I_n point h shifted by e_xshift (xshift < 0: unshifted).
// With m_off >= 0 the source is instead the matrix M of an X M product (TC_APPLY): "row" h is
// row h < a of M (a = the width selected by asel), read from the problem's small workspace at
// byte offset m_off -- complex64 with leading dimension LDR, or complex128 (m_double, rounded to
// complex64) with leading dimension LDM.
template <int KIND>
__global__ void k_xb_prep(Dev D, int xbuf, int xshift, int wsel, unsigned char* xb, long long prob_stride,
                          long long m_off, int m_double, int asel) {
  using K = TcKind<KIND>;
  constexpr int NPL = K::NPL;
  constexpr int EPG = K::TF32 ? 4 : 8;               // elements per 16-byte group
  constexpr int GPC = 64 / EPG;                       // groups per chunk row (all segments)
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  const ProbState& s = D.st[pi];
  if (s.done) return;
  const int w = tc_width(s, p, wsel);
  const int NT = ((2 * w + 15) / 16) * 16;
  const bool msrc = m_off >= 0;
  const int hmax = msrc ? tc_width(s, p, asel) : p.N;   // rows of the source
  const int nc = (hmax + 31) / 32;
  const size_t tile_bytes = (size_t)K::KHALVES * NPL * NT * 128;
  int ldx = 0;
  const float2* X = msrc ? nullptr : tc_buf(D, xbuf, p, ldx);
  const unsigned char* Mb = (const unsigned char*)D.small + p.soff + (msrc ? m_off : 0);
  unsigned char* out = xb + prob_stride * pi;
  const long long total = (long long)nc * NT * GPC;   // (chunk, row, group)
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(q % GPC);
    const long long t = q / GPC;
    const int row = (int)(t % NT);
    const int c = (int)(t / NT);
    const int j = row >> 1;
    const int k0 = g * EPG;                            // K index of the group's first element
    const bool im_block = k0 >= 32;
    const int h0 = 32 * c + (k0 & 31);
    float v[EPG];
#pragma unroll
    for (int e = 0; e < EPG; ++e) {
      const int h = h0 + e;
      float2 x = make_float2(0.f, 0.f);
      if (h < hmax && j < w) {
        if (msrc) {
          if (m_double) {
            const double2 dv = ((const double2*)Mb)[(long long)h * D.L.LDM + j];
            x = make_float2((float)dv.x, (float)dv.y);
          } else {
            x = ((const float2*)Mb)[(long long)h * D.L.LDR + j];
          }
        } else {
          const int hr = xbuf == BUF_Y ? map_row(h, p.n, p.d, p.n + 2, xshift) : h;
          x = X[(long long)j * ldx + hr];
        }
      }
      v[e] = (row & 1) == 0 ? (im_block ? -x.y : x.x) : (im_block ? x.x : x.y);
    }
    uint32_t pw[3][4];                                 // planes x 16 bytes
    if (K::TF32) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t w2[2];
        split_tf32(v[e], w2);
        pw[0][e] = w2[0];
        pw[1][e] = w2[1];
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t w3[3];
        split_pair<NPL>(v[2 * e], v[2 * e + 1], w3);
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) pw[pl][e] = w3[pl];
      }
    }
    const int seg = K::TF32 ? (g >> 3) : 0, gs = K::TF32 ? (g & 7) : g;   // segment, group in the row
    unsigned char* tile = out + (size_t)c * tile_bytes + (size_t)seg * NPL * NT * 128;
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) {
      const int R = pl * NT + row;                     // row within the segment (NT is a multiple of 8)
      *(uint4*)(tile + (size_t)R * 128 + ((gs ^ (R & 7)) << 4)) = make_uint4(pw[pl][0], pw[pl][1], pw[pl][2], pw[pl][3]);
    }
  }
}

// Split planes of the sample grid, table a = part * NPL + plane (part 0: Re, 1: Im), at word
// offset toff + a * Gd4 of the problem.  TF32: one 32-bit word per grid index x.  BF16: 16-bit
// entries in reverse order (entry Gd4 - 1 - x holds sample x; see tc_window), in the first half of
// the table's word range.  One pass per solve.
__device__ __forceinline__ uint16_t bf16_bits(float a) { return (uint16_t)(pack_bf16x2(a, 0.f) & 0xFFFFu); }
__global__ void k_split_tables(Dev D, int tf32) {
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.Gd4; j += gridDim.x * blockDim.x) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const float2* F = (side ? D.gH : D.gF) + p.grid;
      uint32_t* tab = (side ? D.tabH : D.tabF) + p.toff;
      const int x = tf32 ? j : p.Gd4 - 1 - j;
      const float2 v = x < p.Gd ? F[x] : make_float2(0.f, 0.f);
      if (tf32) {
        uint32_t wr[2], wi[2];
        split_tf32(v.x, wr);
        split_tf32(v.y, wi);
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
          tab[(long long)pl * p.Gd4 + x] = wr[pl];
          tab[(long long)(2 + pl) * p.Gd4 + x] = wi[pl];
        }
      } else {
        uint16_t* t16 = (uint16_t*)tab;
        float r[2] = {v.x, v.y};
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          float rest = r[part];
#pragma unroll
          for (int pl = 0; pl < 3; ++pl) {                // x = x0 + x1 + x2, exact for FP32
            const uint16_t h = bf16_bits(rest);
            t16[2LL * (part * 3 + pl) * p.Gd4 + j] = h;
            rest -= __uint_as_float((uint32_t)h << 16);
          }
        }
      }
    }
  }
}

struct TcParams {
  const unsigned char* xb;        // B' tiles (k_xb_prep)
  long long prob_stride;          // bytes of B' tiles per problem
  int adjoint, wsel, ybuf, y_ext;
  int ntbox;                      // B' rows reserved per plane and problem (>= every NT)
  int win_cap;                    // window capacity (entries per table: BF16 a multiple of 8, TF32 of 4)
  int stages;                     // B stages in shared memory (A stages: from the TMEM left by D)
  float* part;                    // split K: one partial tile (ntbox columns x 128 rows) per job
  int* cnt;                       // split K: arrivals per row tile, indexed by its first job (zero between launches)
  long long part_jobs;            // split K: jobs the workspace holds
  // Gram mode (X^* Z of the tall blocks): A' from X (buffer, row shift, width selector), the
  // result into the FP64 small workspace at byte offset out_off, leading dimension out_ld
  int xbuf, xshift, xw;
  long long out_off;
  int out_ld;
};

// Tensor-memory layout of a CTA whose B' tile has NT rows per plane.  With the planes stacked
// along N (NPL * NT <= 256), one MMA per A plane a multiplies A_a by B_0..B_{NPL-1-a} at once
// into D blocks a..NPL-1 (NT columns each), so block k accumulates the products A_a B_b with
// a + b = k: block 0 holds the leading product A_0 B_0 alone and blocks 1.. the corrections,
// each 2^-8 (BF16) or 2^-11 (TF32) smaller than the block before.  The FP32 accumulator rounds
// once per MMA relative to its own magnitude, so the leading block takes one rounding per K step
// instead of NPL, and the corrections' roundings fall below the leading block's.  The epilogue
// adds the blocks from the smallest up.  Otherwise (NPL * NT > 256) every product A_a B_b is its
// own MMA into a single NT-column block.  The A stages follow D.
struct TcLayout {
  bool stacked;
  int dcols, acol0, sa;
};
template <int KIND>
__device__ inline TcLayout tc_layout(int NT) {
  using K = TcKind<KIND>;
  TcLayout t;
  t.stacked = K::NPL * NT <= 256;
  t.dcols = t.stacked ? K::NPL * NT : NT;
  t.acol0 = max(32, (t.dcols + 31) / 32 * 32);
  t.sa = min(TC_MAXSTAGE, (512 - t.acol0) / (K::NPL * K::PCOLS));   // whole-chunk A stages
  return t;
}

// 16 accumulator columns c0..c0+15 of this thread's TMEM lane, the blocks summed from the
// smallest (the last) to the leading one.
template <int NPL>
__device__ __forceinline__ void tc_load_acc(uint32_t taddr, bool stacked, int NT, float* v) {
  uint32_t u[16];
  const int top = stacked ? NPL - 1 : 0;
  tmem_ld_x16(taddr + top * NT, u);
  tmem_ld_wait();
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(u[e]);
  for (int b = top - 1; b >= 0; --b) {
    tmem_ld_x16(taddr + b * NT, u);
    tmem_ld_wait();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] += __uint_as_float(u[e]);
  }
}

// MODE selects what A' is:
//   TC_PRODUCT  the Toeplitz tiles generated from the sample window (above);
//   TC_GRAM     the Gram X^* Z of two tall blocks (N rows, the K dimension): A' row i = conj(X[:, i])
//               read from HBM by the producer warps ([Re x | -Im x] per K chunk, split into planes
//               like the samples), B' = Z by k_xb_prep, one row tile (i < the width of X, at most
//               128), K split over CTAs as for the products; the result goes to the per-problem FP64
//               small workspace;
//   TC_APPLY    the product OUT = X M of a tall block X (N rows, a <= 128 columns, the K dimension)
//               and an a x b matrix M of the small workspace: A' row r = X[r, :] read from HBM
//               ([Re x | Im x] per chunk of 32 columns), B' = M by k_xb_prep, one CTA per row tile
//               and the whole K range (no split), OUT stored like a product.
template <int KIND, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_toeplitz_tc(Dev D, const ToeplitzJob* jobs, TcParams P, int* err) {
  using K = TcKind<KIND>;
  constexpr bool GRAM = MODE == TC_GRAM, APPLY = MODE == TC_APPLY;
  constexpr bool HBMA = GRAM || APPLY;              // A' read from a tall block in HBM, no window
  constexpr int NPL = K::NPL;
  constexpr int NPROD = K::NPROD;
  constexpr int PA[6] = {0, 0, 1, 0, 1, 2};
  constexpr int PB[6] = {0, 1, 0, 2, 1, 0};
  constexpr int GPL = K::TF32 ? 2 : 3;            // planes per part in the global tables
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_win, bar_d;
  __shared__ uint64_t bar_full[TC_MAXSTAGE], bar_empty[TC_MAXSTAGE];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err, s_last;
  __shared__ int ghalf[2 * TC_MAXCH];   // grid offset of each half chunk on one grid line, else -1

  const ToeplitzJob job = jobs[blockIdx.x];
  const ProbDesc& p = D.P[job.prob];
  const ProbState& st = D.st[job.prob];
  if (st.done) return;
  const int w = tc_width(st, p, P.wsel);
  if (w <= 0) return;
  const int aw = HBMA ? tc_width(st, p, P.xw) : 0;   // Gram rows / X M inner dimension: the columns of X
  if (GRAM && (aw <= 0 || aw > TC_BM)) return;
  const int L = P.y_ext ? p.n + 2 : p.n + 1;
  const int rows_total = GRAM ? aw : (P.y_ext ? p.Next : p.N);
  const int row0 = job.mt * TC_BM;
  if (row0 >= rows_total) return;
  if (APPLY && aw <= 0) {                           // X M with an empty X: OUT = 0
    int ldo;
    float2* O = tc_buf(D, P.ybuf, p, ldo);
    const int nr = min(TC_BM, rows_total - row0);
    for (int e = threadIdx.x; e < nr * w; e += blockDim.x) O[(long long)(e / nr) * ldo + row0 + e % nr] = make_float2(0.f, 0.f);
    return;
  }
  const int nc = APPLY ? (aw + 31) / 32 : (p.N + 31) / 32;
  const int cper = (nc + job.nks - 1) / job.nks;
  const int c_begin = job.ks * cper, c_end = min(nc, c_begin + cper);
  const int nchunks = max(0, c_end - c_begin);
  const int NT = ((2 * w + 15) / 16) * 16;
  const TcLayout lay = tc_layout<KIND>(NT);
  // One pipeline stage = one K chunk: its B' tile in shared memory and its A' tile in tensor
  // memory, filled together (full barrier: eight A' warps + the loader's byte count) and
  // released together by one commit of the MMAs that read them.
  const int S = min(P.stages, lay.sa);
  if (nchunks > TC_MAXCH || NT > P.ntbox || S < 1) {   // host sizing rules these out
    if (threadIdx.x == 0) atomicExch(err, 3);
    return;
  }

  // window of grid indices needed by this CTA: [gk(first row) - gh(last h), gk(last row) - gh(first h)],
  // as table entries [wlo, wlo + wlen)
  constexpr int EB = K::TF32 ? 4 : 2;           // bytes per table entry
  int wlo = 0, wlen = 0;
  bool idle = nchunks == 0;                     // an empty K range (a split wider than the problem)
  if (!idle && !HBMA) {
    const int last_row = min(rows_total, row0 + TC_BM) - 1;
    const int h_first = 32 * c_begin, h_last = min(p.N, 32 * c_end) - 1;
    const int f_lo = grid_of_row(row0, L, p) - grid_of_h(h_last, p);
    const int f_hi = grid_of_row(last_row, L, p) - grid_of_h(h_first, p);
    tc_window(!K::TF32, p.Gd4, f_lo, f_hi, wlo, wlen);
    if (wlen > P.win_cap) {
      if (threadIdx.x == 0) atomicExch(err, 3);
      idle = true;
    }
  }
  if (idle && job.nks == 1) return;             // no partial to contribute
  // table a of the problem starts at word toff + a * Gd4 (BF16: its first half, 16-bit entries)
  const unsigned char* gtab = (const unsigned char*)((P.adjoint ? D.tabH : D.tabF) + p.toff);

  // shared memory: B stages (1024-aligned), then the window of the split-plane tables.  A B stage
  // holds KHALVES x NPL x NT rows of 128 bytes: for each 128-byte K segment the planes are
  // stacked with a stride of NT rows, so one descriptor spans B_0 .. B_{NPL-1}.
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const uint32_t stage_bytes = (uint32_t)(K::KHALVES * NPL * P.ntbox) * 128u;
  const uint32_t half_bytes = (uint32_t)(NPL * NT) * 128u;
  unsigned char* Bs = sm;
  unsigned char* wtab = sm + (size_t)P.stages * stage_bytes;   // table a at byte a * win_cap * EB

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    tmem_alloc(&s_tmem, 512);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    mbar_init(&bar_win, 1);
    mbar_init(&bar_d, 1);
    for (int i = 0; i < S; ++i) {
      mbar_init(&bar_full[i], TC_APROD + 1);    // eight A' warps + the loader (with the byte count)
      mbar_init(&bar_empty[i], 1);              // the commit of the stage's MMAs
    }
    s_err = 0;
    s_last = 0;
    fence_barrier_init();
  }
  // grid offset gh of the first of each 16 input points when all 16 lie on one grid line
  for (int idx = threadIdx.x; !HBMA && idx < 2 * nchunks; idx += blockDim.x) {
    const int h0 = 32 * (c_begin + idx / 2) + 16 * (idx & 1);
    const bool line = h0 + 15 < p.N && (h0 % (p.n + 1)) + 15 <= p.n;
    ghalf[idx] = line ? grid_of_h(h0, p) : -1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = s_tmem;

  if (warp == 0) {
    // ------------------------------------------------------------- bulk copies: window and B' stages
    if (lane == 0 && !idle) {
      if (!HBMA) {
        mbar_arrive_expect_tx(&bar_win, (uint32_t)(K::NTAB * wlen * EB));
#pragma unroll
        for (int part = 0; part < 2; ++part)
#pragma unroll
          for (int pl = 0; pl < NPL; ++pl)
            tma_load_1d(wtab + (size_t)(part * NPL + pl) * P.win_cap * EB,
                        gtab + 4LL * (GPL * part + pl) * p.Gd4 + (long long)wlo * EB, (uint32_t)(wlen * EB), &bar_win);
      }
      const uint32_t tile_bytes = (uint32_t)K::KHALVES * half_bytes;
      const unsigned char* src0 = P.xb + P.prob_stride * job.prob + (size_t)c_begin * tile_bytes;
      int issued = 0;
      int s = 0;
      uint32_t ph = 0;                            // stage and round parity (no divisions in the loop)
      for (int it = 0; it < nchunks; ++it) {
        // stage s is free once the MMAs that read its previous contents have completed
        if (it >= S && !mbar_wait_spin(&bar_empty[s], ph ^ 1u, TC_SPIN)) { s_err = 1; break; }
        mbar_arrive_expect_tx(&bar_full[s], tile_bytes);
        tma_load_1d(Bs + (size_t)s * stage_bytes, src0 + (size_t)it * tile_bytes, tile_bytes, &bar_full[s]);
        ++issued;
        if (++s == S) { s = 0; ph ^= 1u; }
      }
      // Tail: the last stages are released by the MMAs that read them, so every copy into this
      // CTA has landed before it exits.
      if (!s_err)
        for (int it = max(0, issued - S); it < issued; ++it)
          if (!mbar_wait_spin(&bar_empty[it % S], (it / S) & 1, TC_SPIN)) { s_err = 1; break; }
      if (!HBMA && !mbar_wait(&bar_win, 0, TC_SPIN)) s_err = 1;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issue
    if (lane == 0 && !idle) {
      uint32_t idesc[NPL];                        // stacked: A_a times B_0..B_{NPL-1-a} into D blocks a..
#pragma unroll
      for (int a = 0; a < NPL; ++a) {
        const int n = lay.stacked ? (NPL - a) * NT : NT;
        idesc[a] = K::TF32 ? idesc_tf32_f32(TC_BM, n) : idesc_bf16_f32(TC_BM, n);
      }
      int s = 0;
      uint32_t ph = 0;
      for (int it = 0; it < nchunks; ++it) {
        if (!mbar_wait_spin(&bar_full[s], ph, TC_SPIN)) {
          s_err = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = tb + lay.acol0 + (uint32_t)s * NPL * K::PCOLS;
        const uint32_t bsm = smem_u32(Bs + (size_t)s * stage_bytes);
        // Operand-major order: all K steps of one MMA shape and operand pair before the next, so
        // consecutive MMAs share their instruction descriptor and operand planes (issuing them
        // K step by K step, with the descriptor or plane changing every MMA, was 2-7 % slower on
        // the products of the C2, C3 and C4 workloads).  Block a of the stacked layout starts with
        // the first MMA of A_0 (which spans every block), so only that one overwrites.
        if (lay.stacked) {
#pragma unroll
          for (int a = 0; a < NPL; ++a)
#pragma unroll
            for (int kk = 0; kk < K::KSTEPS; ++kk) {
              // K step kk: 8 TMEM columns of A; 32 bytes into the 128-byte segment kk / 4 of B
              const uint32_t bseg = bsm + (uint32_t)(kk >> 2) * half_bytes;
              const uint64_t bdk = sdesc_sw128(bseg) + 2 * (kk & 3);
              const uint32_t acc = (a > 0 || it > 0 || kk > 0) ? 1u : 0u;
              mma_ts(K::TF32, tb + (uint32_t)(a * NT), a0 + a * K::PCOLS + 8 * kk, bdk, idesc[a], acc);
            }
        } else {
#pragma unroll
          for (int pr = 0; pr < NPROD; ++pr)
#pragma unroll
            for (int kk = 0; kk < K::KSTEPS; ++kk) {
              const uint32_t bseg = bsm + (uint32_t)(kk >> 2) * half_bytes;
              const uint64_t bd = sdesc_sw128(bseg + (uint32_t)(PB[pr] * NT) * 128u) + 2 * (kk & 3);
              const uint32_t acc = (pr > 0 || it > 0 || kk > 0) ? 1u : 0u;
              mma_ts(K::TF32, tb, a0 + PA[pr] * K::PCOLS + 8 * kk, bd, idesc[0], acc);
            }
        }
        tc_commit(&bar_empty[s]);                 // releases the stage once these MMAs are done
        if (++s == S) { s = 0; ph ^= 1u; }
      }
      tc_commit(&bar_d);                          // arrives when every MMA issued above has completed
    }
  } else {
    // ------------------------------------------------------------- A' producers + epilogue
    // Warps 2..9: quadrant q = warp & 3 (TMEM lanes 32q..32q+31 = tile rows), half hh of every
    // K chunk (input points 32c + 16hh .. +15).
    const int q = warp & 3;
    const int hh = (warp - 2) >> 2;
    const int i = 32 * q + lane;                // row within the tile
    const int row = row0 + i;
    const bool vrow = row < rows_total;
    // window entry of grid index 0 for this row: TF32 entry of grid index g is gk - g... (descending
    // with the input point), BF16 entry is gk + g (ascending, reversed tables)
    const int gk = (HBMA || !vrow) ? 0 : K::TF32 ? grid_of_row(row, L, p) - wlo : p.Gd4 - 1 - grid_of_row(row, L, p) - wlo;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool ok = idle || HBMA || __all_sync(0xffffffffu, mbar_wait(&bar_win, 0, TC_SPIN));
    if (!ok) s_err = 1;
    constexpr int NW = K::TF32 ? 16 : 8;          // words per part and plane: 16 points
    // X M: this lane's row of X (row r of I_n; the box buffer Y holds it at its box row)
    int ldx_a = 0;
    const float2* xrow = nullptr;
    if (APPLY) {
      xrow = tc_buf(D, P.xbuf, p, ldx_a);
      if (vrow) xrow += P.xbuf == BUF_Y ? map_row(row, p.n, p.d, p.n + 2, -1) : row;
    }
    int s = 0;
    uint32_t ph = 0;
    for (int it = 0; ok && it < nchunks; ++it) {
      if (it >= S && !__all_sync(0xffffffffu, mbar_wait_spin(&bar_empty[s], ph ^ 1u, TC_SPIN))) {
        s_err = 1;
        break;
      }
      {
        const int g0 = HBMA ? 0 : ghalf[2 * it + hh];
        // TMEM column of (plane pl, part, point j of this half): BF16 two points per column at
        // pl * 32 + part * 16 + hh * 8 + j / 2; TF32 one point per column at pl * 64 + part * 32 + hh * 16 + j
        const uint32_t a0 = tb + lane_off + lay.acol0 + (uint32_t)s * NPL * K::PCOLS + hh * NW;
        // all table words of the chunk are loaded before the first tensor-memory store (the
        // stores are compiler barriers), so the loads overlap
        uint32_t wv[2][NPL][NW];
        if (APPLY) {
          // A'(r, i) = X[r, i] for the 16 columns i of this half chunk: parts Re x and Im x
          const int i0 = 32 * (c_begin + it) + 16 * hh;
          float v[2][16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const float2 x = (vrow && i0 + jj < aw) ? xrow[(long long)(i0 + jj) * ldx_a] : make_float2(0.f, 0.f);
            v[0][jj] = x.x;
            v[1][jj] = x.y;
          }
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            if (K::TF32) {
#pragma unroll
              for (int e = 0; e < NW; ++e) {
                uint32_t w2[2];
                split_tf32(v[part][e], w2);
                wv[part][0][e] = w2[0];
                wv[part][NPL - 1][e] = w2[1];
              }
            } else {
#pragma unroll
              for (int e = 0; e < NW; ++e) {
                uint32_t w3[3];
                split_pair<NPL>(v[part][2 * e], v[part][2 * e + 1], w3);
#pragma unroll
                for (int pl = 0; pl < NPL; ++pl) wv[part][pl][e] = w3[pl];
              }
            }
          }
        } else if (GRAM) {
          // A'(i, r) = conj(X[r, i]) for the 16 rows r of this half chunk: parts Re x and -Im x
          int ldx = 0;
          const float2* X = tc_buf(D, P.xbuf, p, ldx);   // sets ldx: the column offset is added after
          X += (long long)i * ldx;
          const int r0c = 32 * (c_begin + it) + 16 * hh;
          const bool box = P.xbuf == BUF_Y;
          // on one line of I_n the rows of the box buffer are consecutive too
          const bool line = r0c + 15 < p.N && (r0c % (p.n + 1)) + 15 <= p.n;
          const int rb = (box && line && vrow) ? map_row(r0c, p.n, p.d, p.n + 2, P.xshift) : r0c;
          float v[2][16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int r = r0c + jj;
            float2 x = make_float2(0.f, 0.f);
            if (vrow && r < p.N) x = X[(!box || line) ? rb + jj : map_row(r, p.n, p.d, p.n + 2, P.xshift)];
            v[0][jj] = x.x;
            v[1][jj] = -x.y;
          }
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            if (K::TF32) {
#pragma unroll
              for (int e = 0; e < NW; ++e) {
                uint32_t w2[2];
                split_tf32(v[part][e], w2);
                wv[part][0][e] = w2[0];
                wv[part][NPL - 1][e] = w2[1];
              }
            } else {
#pragma unroll
              for (int e = 0; e < NW; ++e) {
                uint32_t w3[3];
                split_pair<NPL>(v[part][2 * e], v[part][2 * e + 1], w3);
#pragma unroll
                for (int pl = 0; pl < NPL; ++pl) wv[part][pl][e] = w3[pl];
              }
            }
          }
        } else if (g0 >= 0 && K::TF32) {
          // the 16 points lie on one grid line: F(k - h_j) sits at window entry x - j
          const int x = vrow ? gk - g0 : 16;      // rows past the end read nothing (any in-range x)
#pragma unroll
          for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              const uint32_t* T = (const uint32_t*)(wtab + (size_t)(part * NPL + pl) * P.win_cap * EB) + x;
#pragma unroll
              for (int e = 0; e < NW; ++e) wv[part][pl][e] = vrow ? T[-e] : 0u;
            }
        } else if (g0 >= 0) {
          // the 16 points lie on one grid line: point j at window entry x + j (ascending), so the
          // word of the points (2e, 2e + 1) is the 32-bit pair at entry x + 2e -- aligned when x is
          // even, else joined from two aligned words by a 16-bit funnel shift
          const int x = vrow ? gk + g0 : 0;
          const int wb = x >> 1;
          const uint32_t sh = (uint32_t)(x & 1) << 4;
#pragma unroll
          for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              const uint32_t* T = (const uint32_t*)(wtab + (size_t)(part * NPL + pl) * P.win_cap * EB) + wb;
              uint32_t w[NW + 1];
#pragma unroll
              for (int e = 0; e <= NW; ++e) w[e] = vrow ? T[e] : 0u;
#pragma unroll
              for (int e = 0; e < NW; ++e) wv[part][pl][e] = __funnelshift_r(w[e], w[e + 1], sh);
            }
        } else {
          // points on several grid lines: each point from its own table entry
          const int h = 32 * (c_begin + it) + 16 * hh + (lane & 15);
          const int ghl = h < p.N ? grid_of_h(h, p) : INT_MIN;
          int xs[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int g = __shfl_sync(0xffffffffu, ghl, j);
            xs[j] = (vrow && g != INT_MIN) ? (K::TF32 ? gk - g : gk + g) : -1;
          }
#pragma unroll
          for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              const unsigned char* Tb = wtab + (size_t)(part * NPL + pl) * P.win_cap * EB;
#pragma unroll
              for (int e = 0; e < NW; ++e) {
                if (K::TF32) {
                  wv[part][pl][e] = xs[e] >= 0 ? ((const uint32_t*)Tb)[xs[e]] : 0u;
                } else {
                  const uint16_t* T = (const uint16_t*)Tb;
                  const uint32_t lo = xs[2 * e] >= 0 ? (uint32_t)T[xs[2 * e]] : 0u;
                  const uint32_t hi = xs[2 * e + 1] >= 0 ? (uint32_t)T[xs[2 * e + 1]] << 16 : 0u;
                  wv[part][pl][e] = lo | hi;
                }
              }
            }
        }
#pragma unroll
        for (int part = 0; part < 2; ++part)
#pragma unroll
          for (int pl = 0; pl < NPL; ++pl) {
            const uint32_t col = a0 + pl * K::PCOLS + part * (K::PCOLS / 2);
            if (K::TF32) tmem_st_x16(col, wv[part][pl]);
            else tmem_st_x8(col, wv[part][pl]);
          }
        tmem_st_wait();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_full[s]);
      if (++s == S) { s = 0; ph ^= 1u; }
    }
    // epilogue: D (TMEM) -> Y; the two warps of a quadrant take alternate 16-column groups
    const bool dready = idle || __all_sync(0xffffffffu, mbar_wait(&bar_d, 0, TC_SPIN));
    if (!dready) s_err = 1;
    int ldy;
    float2* Y = GRAM ? nullptr : tc_buf(D, P.ybuf, p, ldy);
    double2* G = GRAM ? (double2*)(D.small + p.soff + P.out_off) : nullptr;
    // output entry (row, column j): Y[j][row] of the product, or Gram entry (row, j) in FP64
    auto store = [&](int j, float re, float im) {
      if (GRAM) G[(long long)row * P.out_ld + j] = make_double2((double)re, (double)im);
      else Y[(long long)j * ldy + row] = make_float2(re, im);
    };
    if (job.nks == 1) {
      if (dready && !s_err) {
        tc_fence_after();
        for (int c0 = 16 * hh; c0 < NT; c0 += 32) {
          float v[16];
          tc_load_acc<NPL>(tb + lane_off + c0, lay.stacked, NT, v);
          if (vrow) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int j = c0 / 2 + e;
              if (j < w) store(j, v[2 * e], v[2 * e + 1]);
            }
          }
        }
      }
    } else {
      // split K: this CTA's partial tile (zeros for an empty K range) into its slot, column-major
      // (coalesced over the rows of a warp); then one arrival on the tile's counter
      const size_t slot = (size_t)P.ntbox * TC_BM;
      float* mine = P.part + (size_t)blockIdx.x * slot;
      const bool mine_ok = ws_ok(D, (long long)blockIdx.x - job.ks + job.nks <= P.part_jobs && job.ks < job.nks, 21);
      if (dready && !s_err && !idle) tc_fence_after();
      for (int c0 = 16 * hh; c0 < NT; c0 += 32) {
        float v[16];
        if (dready && !s_err && !idle) {
          tc_load_acc<NPL>(tb + lane_off + c0, lay.stacked, NT, v);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0.f;
        }
        if (mine_ok) {
#pragma unroll
          for (int e = 0; e < 16; ++e) mine[(size_t)(c0 + e) * TC_BM + i] = v[e];
        }
      }
      __threadfence();
      named_bar_sync(1, 32 * TC_APROD);
      const int first_job = blockIdx.x - job.ks;  // the tile's CTAs are consecutive jobs
      if (warp == 2 && lane == 0) s_last = mine_ok && atomicAdd(&P.cnt[first_job], 1) == job.nks - 1;
      named_bar_sync(1, 32 * TC_APROD);
      if (s_last) {
        // every other CTA of the tile has stored its partial (fence before its arrival): add the
        // partials in the order of their K ranges -- in FP32 for a product (at most 16 ranges;
        // dependent FP64 additions are slow here), in FP64 for a Gram (up to hundreds of ranges)
        __threadfence();
        const float* base = P.part + (size_t)first_job * slot;
        using Acc = typename std::conditional<GRAM, double, float>::type;
        for (int c0 = 16 * hh; c0 < NT; c0 += 32) {
          Acc v[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = (Acc)__ldcg(base + (size_t)(c0 + e) * TC_BM + i);
          for (int k = 1; k < job.nks; ++k) {
            const float* src = base + (size_t)k * slot + (size_t)c0 * TC_BM + i;
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] += (Acc)__ldcg(src + (size_t)e * TC_BM);
          }
          if (vrow) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int j = c0 / 2 + e;
              if (j < w) {
                if (GRAM) G[(long long)row * P.out_ld + j] = make_double2(v[2 * e], v[2 * e + 1]);
                else store(j, (float)v[2 * e], (float)v[2 * e + 1]);
              }
            }
          }
        }
        if (warp == 2 && lane == 0) P.cnt[first_job] = 0;   // ready for the next launch
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_err && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 0) {
    tc_fence_after();
    // on an error path, let the MMAs already issued finish before the columns are released
    if (s_err && !idle) mbar_wait(&bar_d, 0, TC_SPIN);
    tmem_dealloc(tb, 512);
  }
}

}  // namespace

// ----------------------------------------------------------------------------- host side
int tc_planes(int kind) { return kind == PRONY_BF16X3 ? 3 : 2; }
size_t tc_stage_bytes(int kind, int ntbox) { return (size_t)(kind == PRONY_TF32X3 ? 2 : 1) * tc_planes(kind) * ntbox * 128; }
size_t tc_elem_bytes(int kind) { return kind == PRONY_TF32X3 ? 4 : 2; }

size_t tc_entry_bytes(int kind) { return kind == PRONY_TF32X3 ? 4 : 2; }
size_t tc_smem_bytes(int kind, int ntbox, int stages, int win_cap) {
  return 1024 + (size_t)stages * tc_stage_bytes(kind, ntbox) + (size_t)2 * tc_planes(kind) * win_cap * tc_entry_bytes(kind);
}

void launch_split_tables(const Dev& D, int kind, cudaStream_t s) {
  note_launch();
  dim3 g(blocks_per_problem(std::min((D.maxGd + 3) / 4 / 256 + 1, 64), D.nprob), D.nprob);
  k_split_tables<<<g, 256, 0, s>>>(D, kind == PRONY_TF32X3 ? 1 : 0);
}

// Bytes of B' tiles reserved per problem: every chunk at the widest tile of the batch.
long long tc_prob_stride(int kind, int ntbox, int maxnc) { return (long long)maxnc * (long long)tc_stage_bytes(kind, ntbox); }

static void xb_prep(const Dev& D, int xbuf, int xshift, int wsel, void* xb, int kind, long long prob_stride,
                    long long m_off, int m_double, int asel, long long src_rows, cudaStream_t s) {
  note_launch();
  // items (chunk, row, 16-byte group) of the largest problem, about four per thread
  const long long items = (long long)((src_rows + 31) / 32) * (2 * D.maxR0 + 16) * 16;
  dim3 g(blocks_per_problem(std::min<long long>(1024, (items + 1023) / 1024), D.nprob), D.nprob);
  unsigned char* b = (unsigned char*)xb;
  switch (kind) {
    case PRONY_BF16X3:
      k_xb_prep<PRONY_BF16X3><<<g, 256, 0, s>>>(D, xbuf, xshift, wsel, b, prob_stride, m_off, m_double, asel);
      break;
    case PRONY_BF16X2:
      k_xb_prep<PRONY_BF16X2><<<g, 256, 0, s>>>(D, xbuf, xshift, wsel, b, prob_stride, m_off, m_double, asel);
      break;
    default:
      k_xb_prep<PRONY_TF32X3><<<g, 256, 0, s>>>(D, xbuf, xshift, wsel, b, prob_stride, m_off, m_double, asel);
      break;
  }
}

void launch_xb_prep(const Dev& D, int xbuf, int xshift, int wsel, void* xb, int kind, long long prob_stride,
                    cudaStream_t s) {
  xb_prep(D, xbuf, xshift, wsel, xb, kind, prob_stride, -1, 0, 0, D.maxN, s);
}

template <int KIND, int MODE>
static cudaError_t launch_tc_kind(const Dev& D, const ToeplitzJob* jobs, int njobs, const TcParams& P, int* err,
                                  size_t sm, cudaStream_t s) {
  static size_t set = 0;
  if (sm > set) {
    // the attribute must cover this launch's dynamic shared memory (static + dynamic <= 227 KB)
    cudaError_t e =
        cudaFuncSetAttribute(k_toeplitz_tc<KIND, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    set = sm;
  }
  k_toeplitz_tc<KIND, MODE><<<njobs, TC_THREADS, sm, s>>>(D, jobs, P, err);
  return cudaGetLastError();
}

size_t tc_part_floats(int ntbox) { return (size_t)ntbox * TC_BM; }

cudaError_t launch_toeplitz_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int adjoint, int wsel, int ybuf,
                               int y_ext, int kind, int ntbox, int win_cap, int stages, const void* xb,
                               long long prob_stride, float* part, int* cnt, long long part_jobs, int* err,
                               cudaStream_t s) {
  TcParams P{(const unsigned char*)xb, prob_stride, adjoint, wsel, ybuf, y_ext, ntbox, win_cap, stages, part, cnt,
             part_jobs, 0, -1, 0, 0, 0};
  const size_t sm = tc_smem_bytes(kind, ntbox, stages, win_cap);
  note_launch();
  switch (kind) {
    case PRONY_BF16X3: return launch_tc_kind<PRONY_BF16X3, TC_PRODUCT>(D, jobs, njobs, P, err, sm, s);
    case PRONY_BF16X2: return launch_tc_kind<PRONY_BF16X2, TC_PRODUCT>(D, jobs, njobs, P, err, sm, s);
    default: return launch_tc_kind<PRONY_TF32X3, TC_PRODUCT>(D, jobs, njobs, P, err, sm, s);
  }
}

// The Gram X^* Z of two tall blocks on the tensor cores in three BF16 planes (B' tiles of Z from
// k_xb_prep at `xb`), one CTA per problem and K range (jobs: row tile 0).
cudaError_t launch_gram_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int xbuf, int xshift, int xw, int zw,
                           long long out_off, int out_ld, int ntbox, int stages, const void* xb, long long prob_stride,
                           float* part, int* cnt, long long part_jobs, int* err, cudaStream_t s) {
  TcParams P{(const unsigned char*)xb, prob_stride, 0, zw, 0, 0, ntbox, 0, stages, part, cnt, part_jobs,
             xbuf, xshift, xw, out_off, out_ld};
  const size_t sm = tc_smem_bytes(PRONY_BF16X3, ntbox, stages, 0);
  note_launch();
  return launch_tc_kind<PRONY_BF16X3, TC_GRAM>(D, jobs, njobs, P, err, sm, s);
}

// OUT = X M for every live problem on the tensor cores in three BF16 planes: B' tiles of M (small
// workspace at m_off) by k_xb_prep, then one CTA per row tile of N rows (jobs with nks = 1).
cudaError_t launch_apply_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int xbuf, int xw, int outw,
                            long long m_off, int m_double, int outbuf, int ntbox, int stages, void* xb,
                            long long prob_stride, int* err, cudaStream_t s) {
  xb_prep(D, -1, -1, outw, xb, PRONY_BF16X3, prob_stride, m_off, m_double, xw, D.maxR0, s);
  TcParams P{(const unsigned char*)xb, prob_stride, 0, outw, outbuf, 0, ntbox, 0, stages, nullptr, nullptr, 0,
             xbuf, -1, xw, 0, 0};
  // at least half the shared memory of an SM, so that one CTA holds an SM (and all of its tensor
  // memory) at a time
  const size_t sm = std::max<size_t>(tc_smem_bytes(PRONY_BF16X3, ntbox, stages, 0), 116 * 1024);
  note_launch();
  return launch_tc_kind<PRONY_BF16X3, TC_APPLY>(D, jobs, njobs, P, err, sm, s);
}
