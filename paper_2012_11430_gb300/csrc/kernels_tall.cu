// Data-parallel kernels over the rows of one or many problems: grid preparation,
// Philox starting block, tall-skinny Gram and products of the block power method
// (Algorithm 3), the Vandermonde right-hand side conj(A) f and the LS residual
// (Eq. ls_probl), and the exponential sum of Eq. 1 with its vector-Jacobian product.
#include "common.cuh"

#include <algorithm>
#include <map>

namespace {

__device__ inline const ProbDesc& prob(const Dev& D, int p) { return D.P[p]; }

__device__ inline float2* buf_base(const Dev& D, int buf, const ProbDesc& p, int& ld) {
  switch (buf) {
    case BUF_V: ld = p.N; return D.V + p.xoff;
    case BUF_U: ld = p.N; return D.U + p.xoff;
    case BUF_B1: ld = p.N; return D.B1 + p.xoff;
    case BUF_B2: ld = p.N; return D.B2 + p.xoff;
    default: ld = p.Next; return D.Y + p.yoff;
  }
}

__device__ inline int width_of(const ProbState& s, const ProbDesc& p, int sel) { return sel_width(s, p, sel); }

// Row of buffer `buf` holding row r of I_n (Y is laid out over the box {0..n+1}^d).
__device__ inline int buf_row(int buf, const ProbDesc& p, int r, int shift) {
  return buf == BUF_Y ? map_row(r, p.n, p.d, p.n + 2, shift) : r;
}

template <typename T>
__device__ inline T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x < 32) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : (T)0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// ----------------------------------------------------------------------------- grid prep
__global__ void k_state_init(Dev D) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.nprob) return;
  ProbState s = {};
  s.wu = D.P[p].r0;
  s.wv = D.P[p].r0;
  s.rank_det = -1;
  s.rank_used = D.P[p].m;
  s.resid2_prev = -1.0;
  D.st[p] = s;
}

// gF = f, gH(x) = conj f(-x) (zero where -x leaves the grid); ||T||_F^2 by the
// multiplicity of each difference (prod_l (n+1-|x_l|)), ||f||^2 over I_n, finiteness.
__global__ void k_prep(Dev D) {
  __shared__ double sh[32];
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  double accT = 0.0, accF = 0.0;
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.Gd; i += gridDim.x * blockDim.x) {
    int rem = i, mir = 0, mul = 1;
    double w = 1.0;
    bool inT = true, inI = true, mvalid = true;
    for (int l = p.d - 1; l >= 0; --l) {
      int dig = rem % p.G;
      rem /= p.G;
      int x = dig - p.n;
      int ax = x < 0 ? -x : x;
      if (ax > p.n) inT = false; else w *= (double)(p.n + 1 - ax);
      if (x < 0 || x > p.n) inI = false;
      int md = 2 * p.n - dig;  // digit of -x
      if (md < 0) mvalid = false;
      mir += md * mul;
      mul *= p.G;
    }
    double2 f = D.grid64[p.grid + i];
    if (!isfinite(f.x) || !isfinite(f.y)) bad = 1;
    D.gF[p.grid + i] = make_float2((float)f.x, (float)f.y);
    float2 h = make_float2(0.f, 0.f);
    if (mvalid) {
      double2 fm = D.grid64[p.grid + mir];
      h = make_float2((float)fm.x, -(float)fm.y);
    }
    D.gH[p.grid + i] = h;
    double a2 = f.x * f.x + f.y * f.y;
    if (inT) accT += w * a2;
    if (inI) accF += a2;
  }
  double sT = block_sum(accT, sh);
  double sF = block_sum(accF, sh);
  if (bad) atomicOr(&D.st[pi].nonfinite, 1);
  // block sums in fixed block order
  double2* slot = (double2*)red_region(D, pi);
  if (threadIdx.x == 0 && ws_ok(D, 16LL * (blockIdx.x + 1) <= D.red_stride, 11)) slot[blockIdx.x] = make_double2(sT, sF);
  if (red_arrive(D, pi, gridDim.x) && threadIdx.x == 0) {
    double t2 = 0.0, f2 = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const double2 v = __ldcg(slot + b);
      t2 += v.x;
      f2 += v.y;
    }
    D.st[pi].normT2 = t2;
    D.st[pi].normf2 = f2;
  }
}

// V_0 entry (i, j) = complex normal from Philox counter i*r0 + j (Algorithm 3 start block).
__global__ void k_init_v0(Dev D, unsigned long long seed) {
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  // a thread takes rows, the threads of a warp neighbouring rows of one column at a time
  // (coalesced stores); the counter of entry (row, col) is row * r0 + col
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < p.N; row += gridDim.x * blockDim.x)
  for (int col = 0; col < p.r0; ++col) {
    const long long q = (long long)row * p.r0 + col;
    uint64_t c[4] = {(uint64_t)q, 0, 0, 0};
    philox4x64(c, seed, PRONY_STREAM_V0);
    float u0 = (float)philox_u01(c[0]), u1 = (float)philox_u01(c[1]);
    float r = sqrtf(-logf(u0)), sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    D.V[p.xoff + (long long)col * p.N + row] = make_float2(r * cs, r * sn);
  }
}

// Clears a block of the small workspace of every problem still iterating (a stopped problem keeps
// the Q and U^* T_l V of its last iteration).
__global__ void k_zero_small(Dev D, long long off, long long bytes) {
  if (D.st[blockIdx.y].done) return;
  const ProbDesc& p = D.P[blockIdx.y];
  unsigned int* b = (unsigned int*)(D.small + p.soff + off);
  for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < bytes / 4; i += gridDim.x * blockDim.x) b[i] = 0u;
}

// ----------------------------------------------------------------------------- tall-skinny Gram
// out[a][b] += sum_r conj(X[r, a]) Z[r, b] over a block of `chunk` rows (chosen by the launcher
// so that the batch gives a few blocks per SM: few blocks per problem means few FP64 atomics on
// the same output entries).
//
// Rows are staged RS at a time in two alternating shared-memory buffers (RS = 64 down to 8: the
// most that the staged columns of this problem leave room for): each thread loads the next rows'
// values into registers while the current ones are multiplied, then stores them.  A thread stages one row (its row index is computed once per
// pass) and several columns; the values are stored column-major with a row pitch of RS + 1 and
// pre-arranged for paired FP32 FMAs (fma.rn.f32x2): x as (Re x, Re x, Im x, Im x) and z as
// (Re z, Im z, Im z, -Re z), so that conj(x) z is two paired FMAs on (re, im) accumulators.
// Output ownership is interleaved: thread (ti, tj) owns the entries (ti + NA i, tj + NB j),
// i, j < 4, so the threads of a warp read consecutive columns (different banks) or the same one
// (broadcast).  When there are fewer 4x4 tiles than threads, threads split the staged rows into
// row groups whose partial sums are added in shared memory; when there are more, the tiles are
// processed in batches (every batch re-stages the rows).  Each block stores its partial Gram; the
// last block of the problem adds the partials (FP32, a fixed order) into the FP64 output.
constexpr int GRAM_T = 4;           // register tile (GRAM_T x GRAM_T complex accumulators)
constexpr int GRAM_KMAX = 10;       // staged values per thread and pass: (a + b) RS <= 256 GRAM_KMAX

__host__ __device__ inline int gram_rows(int LR) { return LR <= 40 ? 32 : LR <= 80 ? 16 : 8; }
// float4 entries of one staging buffer (sized by the widest blocks of the batch, LR columns)
__host__ __device__ inline int gram_buf_elems(int LR) { return 2 * LR * (gram_rows(LR) + 1); }
// Rows staged per pass for a block of `cols` staged columns (float4 each) of which `loaded` are
// read from HBM: the most (64, 32, 16, 8) that fit the buffer and the staging registers.
__device__ inline int gram_rows_for(int cols, int loaded, int LR) {
  const int cap = gram_buf_elems(LR);
  int rs = 64;
  while (rs > 8 && (cols * (rs + 1) > cap || loaded * rs > 256 * 10)) rs >>= 1;
  return rs;
}

__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return make_float2(lo, hi);
}
__device__ __forceinline__ void ffma2(unsigned long long& acc, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

__global__ void __launch_bounds__(256, 2) k_gram(Dev D, int xbuf, int xshift, int xw, int zbuf, int zshift, int zw,
                                              long long out_off, int out_ld, int chunk) {
  extern __shared__ float4 smem4[];
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  const ProbState& s = D.st[pi];
  if (s.done) return;
  const int a = width_of(s, p, xw), b = width_of(s, p, zw);
  const int r_begin = blockIdx.x * chunk;
  if (r_begin >= p.N || a <= 0 || b <= 0) return;
  const int r_end = min(p.N, r_begin + chunk);
  const int LR = D.L.LDR;
  // X^* X (same buffer, shift and width): the rows are loaded once and only the tiles on and
  // above the diagonal are computed, the others written as their conjugate mirrors
  const bool sym = xbuf == zbuf && xshift == zshift && a == b;
  // staged columns: a of X, then b of Z (for X^* X the second form of the same a columns)
  const int ZC = a;                                // first staged column of Z
  const int RS = gram_rows_for(a + b, sym ? a : a + b, LR), PR = RS + 1;
  const size_t buf_elems = (size_t)gram_buf_elems(LR);   // X then Z, column-major with row pitch PR
  // [RG-1][per_batch][16] packed partial sums, over the staging buffers once the rows are done
  unsigned long long* red = (unsigned long long*)smem4;
  int ldx, ldz;
  const float2* X = buf_base(D, xbuf, p, ldx);
  const float2* Z = buf_base(D, zbuf, p, ldz);
  const int NA = (a + GRAM_T - 1) / GRAM_T, NB = (b + GRAM_T - 1) / GRAM_T;
  const int ntile = sym ? NA * (NA + 1) / 2 : NA * NB;
  const int nthr = blockDim.x;
  const int per_batch = min(ntile, nthr);
  const int RG = max(1, min(RS, nthr / per_batch));    // row groups (1 when tiles >= threads)
  const int nbatch = (ntile + per_batch - 1) / per_batch;
  double2* out = (double2*)(D.small + p.soff + out_off);
  float2* mine = (float2*)red_region(D, pi) + (size_t)blockIdx.x * a * b;   // this block's partial Gram
  const bool mine_ok = ws_ok(D, 8LL * a * b * (blockIdx.x + 1) <= D.red_stride, 12);
  // staging role: one row, columns c0, c0 + cstep, ... (k-th: X column if below a, else Z)
  const int my_rr = threadIdx.x % RS, c0 = threadIdx.x / RS, cstep = nthr / RS;
  float2 held[GRAM_KMAX];
  auto load_rows = [&](int r0) {
    const int r = r0 + my_rr;
    const bool ok = r < r_end;
    const int gx = ok ? buf_row(xbuf, p, r, xshift) : 0, gz = ok ? buf_row(zbuf, p, r, zshift) : 0;
    const int ncols = sym ? a : a + b;
#pragma unroll
    for (int k = 0; k < GRAM_KMAX; ++k) {
      const int col = c0 + k * cstep;
      float2 v = make_float2(0.f, 0.f);
      if (ok && col < ncols) v = col < a ? X[(long long)col * ldx + gx] : Z[(long long)(col - a) * ldz + gz];
      held[k] = v;
    }
  };
  auto store_rows = [&](int buf) {
    float4* Xs = smem4 + (size_t)buf * buf_elems;
#pragma unroll
    for (int k = 0; k < GRAM_KMAX; ++k) {
      const int col = c0 + k * cstep;
      const float2 v = held[k];
      // X and Z regions are contiguous: Z column c sits at column ZC + c of the buffer
      if (col < a) {
        Xs[col * PR + my_rr] = make_float4(v.x, v.x, v.y, v.y);
        if (sym) Xs[(col + ZC) * PR + my_rr] = make_float4(v.x, v.y, v.y, -v.x);
      } else if (!sym && col < a + b) {
        Xs[(col - a + ZC) * PR + my_rr] = make_float4(v.x, v.y, v.y, -v.x);
      }
    }
  };
  for (int batch = 0; batch < nbatch; ++batch) {
    const int tile = batch * per_batch + threadIdx.x % per_batch, grp = threadIdx.x / per_batch;
    const bool active = grp < RG && tile < ntile;
    int ti = tile / NB, tj = tile % NB;
    if (sym) {                                    // tile -> (ti, tj), ti <= tj, row by row
      ti = 0;
      int rest = min(tile, ntile - 1);
      while (rest >= NA - ti) {
        rest -= NA - ti;
        ++ti;
      }
      tj = ti + rest;
    }
    // offsets of the owned columns in a buffer (entries past a or b read a valid column; their
    // sums are never stored)
    int xo[GRAM_T], zo[GRAM_T];
#pragma unroll
    for (int i = 0; i < GRAM_T; ++i) {
      xo[i] = min(ti + NA * i, a - 1) * PR;
      zo[i] = (min(tj + NB * i, b - 1) + ZC) * PR;
    }
    unsigned long long acc[GRAM_T][GRAM_T];
#pragma unroll
    for (int i = 0; i < GRAM_T; ++i)
#pragma unroll
      for (int j = 0; j < GRAM_T; ++j) acc[i][j] = 0ull;
    __syncthreads();                              // the buffers are free (previous batch done)
    load_rows(r_begin);
    store_rows(0);
    int k = 0;
    for (int r0 = r_begin; r0 < r_end; r0 += RS, k ^= 1) {
      const bool more = r0 + RS < r_end;
      if (more) load_rows(r0 + RS);               // in flight while these rows are multiplied
      __syncthreads();
      // each staged value is 16 bytes read as two packed pairs: x = ((Re x, Re x), (Im x, Im x)),
      // z = ((Re z, Im z), (Im z, -Re z))
      const ulonglong2* Bs = (const ulonglong2*)(smem4 + (size_t)k * buf_elems);
      if (active) {
        const int nrows = min(RS, r_end - r0);
        for (int rr = grp; rr < nrows; rr += RG) {
          ulonglong2 xa[GRAM_T], zb[GRAM_T];
#pragma unroll
          for (int i = 0; i < GRAM_T; ++i) xa[i] = Bs[xo[i] + rr];
#pragma unroll
          for (int j = 0; j < GRAM_T; ++j) zb[j] = Bs[zo[j] + rr];
#pragma unroll
          for (int i = 0; i < GRAM_T; ++i)
#pragma unroll
            for (int j = 0; j < GRAM_T; ++j) {
              ffma2(acc[i][j], xa[i].x, zb[j].x);   // (Re x Re z, Re x Im z)
              ffma2(acc[i][j], xa[i].y, zb[j].y);   // + (Im x Im z, -Im x Re z)
            }
        }
      }
      if (more) store_rows(k ^ 1);                // the other buffer was released by the sync above
    }
    // row groups: partial sums meet in shared memory, group 0 adds them (fixed order)
    if (RG > 1) {
      __syncthreads();                            // every group is done with the staged rows
      if (active && grp > 0) {
        unsigned long long* dst = red + ((size_t)(grp - 1) * per_batch + (tile - batch * per_batch)) * 16;
#pragma unroll
        for (int i = 0; i < GRAM_T; ++i)
#pragma unroll
          for (int j = 0; j < GRAM_T; ++j) dst[i * GRAM_T + j] = acc[i][j];
      }
      __syncthreads();
      if (active && grp == 0) {
        for (int g = 1; g < RG; ++g) {
          const unsigned long long* src = red + ((size_t)(g - 1) * per_batch + (tile - batch * per_batch)) * 16;
#pragma unroll
          for (int i = 0; i < GRAM_T; ++i)
#pragma unroll
            for (int j = 0; j < GRAM_T; ++j) {
              const float2 u = upk2(acc[i][j]), v = upk2(src[i * GRAM_T + j]);
              acc[i][j] = pk2(u.x + v.x, u.y + v.y);
            }
        }
      }
    }
    if (active && grp == 0) {
#pragma unroll
      for (int i = 0; i < GRAM_T; ++i)
#pragma unroll
        for (int j = 0; j < GRAM_T; ++j) {
          const int ia = ti + NA * i, jb = tj + NB * j;
          if (ia < a && jb < b) {
            const float2 v = upk2(acc[i][j]);
            if (mine_ok) {
              mine[ia * b + jb] = v;
              if (sym && ti != tj) mine[jb * b + ia] = make_float2(v.x, -v.y);   // mirror of a tile above the diagonal
            }
          }
        }
    }
  }
  // The blocks' partial Grams (one slot of a x b each) added in FP32 in a fixed order: slot k
  // goes to the partial sum k mod 4 of its entry, and the four are combined pairwise.  Each thread
  // takes GR entries at a time, so that 4 GR loads are in flight.  (FP32 sums of at most 64
  // partials add less rounding than each partial already carries from its own rows; FP64
  // additions, at a small fraction of the FP32 rate here, made this one block per problem the
  // longest part of the launch.)
  const int nblk = (p.N + chunk - 1) / chunk;
  if (red_arrive(D, pi, nblk)) {
    constexpr int GR = 2;
    const float2* slots = (const float2*)red_region(D, pi);
    const int ss = a * b;
    for (int e0 = threadIdx.x; e0 < ss; e0 += GR * blockDim.x) {
      float2 acc[GR][4];
#pragma unroll
      for (int g = 0; g < GR; ++g)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[g][u] = make_float2(0.f, 0.f);
      int k = 0;
      for (; k + 4 <= nblk; k += 4) {
        float2 v[GR][4];
#pragma unroll
        for (int g = 0; g < GR; ++g)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e0 + g * blockDim.x;
            v[g][u] = e < ss ? __ldcg(slots + (size_t)(k + u) * ss + e) : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int g = 0; g < GR; ++g)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            acc[g][u].x += v[g][u].x;
            acc[g][u].y += v[g][u].y;
          }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {                 // the last nblk mod 4 slots
        if (k + u < nblk) {
#pragma unroll
          for (int g = 0; g < GR; ++g) {
            const int e = e0 + g * blockDim.x;
            const float2 v = e < ss ? __ldcg(slots + (size_t)(k + u) * ss + e) : make_float2(0.f, 0.f);
            acc[g][u].x += v.x;
            acc[g][u].y += v.y;
          }
        }
      }
#pragma unroll
      for (int g = 0; g < GR; ++g) {
        const int e = e0 + g * blockDim.x;
        if (e < ss) {
          const float tx = (acc[g][0].x + acc[g][1].x) + (acc[g][2].x + acc[g][3].x);
          const float ty = (acc[g][0].y + acc[g][1].y) + (acc[g][2].y + acc[g][3].y);
          double2* o = &out[(e / b) * out_ld + e % b];
          *o = make_double2(o->x + (double)tx, o->y + (double)ty);
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------- X M products
// OUT[r, j] = sum_i X[r, i] M[i][j] (- Z[r, j] with OUT = Z - X M for the residual).  A block
// takes `rows` rows (128, or 64 when the blocks are wide), stages them and M in shared memory
// once, then each thread computes one row and four columns at a time (one X value and four
// broadcast M values per four complex products).  X and OUT may be the same buffer: every
// block reads its rows before writing them.
__global__ void __launch_bounds__(256) k_apply(Dev D, int xbuf, int xw, int outw, long long m_off, int m_double,
                                               int zbuf, int outbuf, int norm_only, int rows) {
  extern __shared__ float2 smem[];
  __shared__ double shr[32];
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  ProbState& s = D.st[pi];
  if (s.done) return;
  const int a = width_of(s, p, xw), b = width_of(s, p, outw);
  const int r0 = blockIdx.x * rows;
  if (r0 >= p.N || b <= 0) return;
  const int ldm = (b + 3) & ~3;                   // M rows padded to whole groups of four columns
  float2* Ms = smem;                              // [a][ldm]
  float2* Xs = smem + (size_t)D.L.LDR * ((D.L.LDR + 3) & ~3);   // [a][rows]
  for (int idx = threadIdx.x; idx < a * ldm; idx += blockDim.x) {
    const int i = idx / ldm, j = idx % ldm;
    float2 v = make_float2(0.f, 0.f);
    if (j < b) {
      if (m_double) {
        const double2 dv = ((const double2*)(D.small + p.soff + m_off))[i * D.L.LDM + j];
        v = make_float2((float)dv.x, (float)dv.y);
      } else {
        v = ((const float2*)(D.small + p.soff + m_off))[i * D.L.LDR + j];
      }
    }
    Ms[idx] = v;
  }
  int ldx;
  const float2* X = buf_base(D, xbuf, p, ldx);
  // a thread stages one row (blockDim.x is a multiple of rows) and every cstep-th column, eight
  // loads in flight at a time
  const int rr = threadIdx.x % rows, cg = threadIdx.x / rows;
  const int ngrp = blockDim.x / rows;
  const int r = r0 + rr;
  {
    const bool ok = r < p.N;
    const int gx = ok ? buf_row(xbuf, p, r, -1) : 0;
    for (int cb = cg; cb < a; cb += 8 * ngrp) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = cb + u * ngrp;
        v[u] = (ok && col < a) ? X[(long long)col * ldx + gx] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = cb + u * ngrp;
        if (col < a) Xs[col * rows + rr] = v[u];
      }
    }
  }
  __syncthreads();
  int ldz = 0, ldo = 0;
  const float2* Z = zbuf >= 0 ? buf_base(D, zbuf, p, ldz) : nullptr;
  float2* O = norm_only ? nullptr : buf_base(D, outbuf, p, ldo);
  // squares of a row summed in FP32 (the entries are FP32 values; b <= 128 terms), blocks in FP64
  float nrm = 0.f;
  if (r < p.N) {
    const int gz = Z ? buf_row(zbuf, p, r, -1) : 0;
    const int go = O ? buf_row(outbuf, p, r, -1) : 0;
    for (int j0 = 4 * cg; j0 < b; j0 += 4 * ngrp) {
      float2 zv[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)      // issued before the products so that their latency overlaps them
        zv[e] = (Z && j0 + e < b) ? Z[(long long)(j0 + e) * ldz + gz] : make_float2(0.f, 0.f);
      // x m as paired FP32 FMAs on M as stored: p1 += (Re x, Re x)(Re m, Im m),
      // p2 += (Im x, Im x)(Re m, Im m); then x m = (p1.x - p2.y, p1.y + p2.x)
      unsigned long long p1[4] = {0ull, 0ull, 0ull, 0ull}, p2[4] = {0ull, 0ull, 0ull, 0ull};
      for (int i = 0; i < a; ++i) {
        const float2 x = Xs[i * rows + rr];
        const unsigned long long xr = pk2(x.x, x.x), xi = pk2(x.y, x.y);
        const unsigned long long* mrow = (const unsigned long long*)(Ms + i * ldm + j0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const unsigned long long mm = mrow[e];
          ffma2(p1[e], xr, mm);
          ffma2(p2[e], xi, mm);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = j0 + e;
        if (j >= b) break;
        const float2 q1 = upk2(p1[e]), q2 = upk2(p2[e]);
        float2 v = make_float2(q1.x - q2.y, q1.y + q2.x);
        if (Z) {
          v.x = zv[e].x - v.x;
          v.y = zv[e].y - v.y;
        }
        if (norm_only) nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
        else O[(long long)j * ldo + go] = v;
      }
    }
  }
  if (norm_only) {
    double t = block_sum((double)nrm, shr);
    double* slot = (double*)red_region(D, pi);
    if (threadIdx.x == 0 && ws_ok(D, 8LL * (blockIdx.x + 1) <= D.red_stride, 13)) slot[blockIdx.x] = t;
    const int nblk = (p.N + rows - 1) / rows;
    if (red_arrive(D, pi, nblk)) {
      // the block sums in a fixed order: thread i adds slots i, i + 256, ..., then a block sum
      double r2 = 0.0;
      for (int k = threadIdx.x; k < nblk; k += blockDim.x) r2 += __ldcg(slot + k);
      r2 = block_sum(r2, shr);
      if (threadIdx.x == 0) s.resid2 = r2;
    }
  }
}

// Largest-modulus row of each of the first m columns (lowest row on ties).
__global__ void k_argmax(Dev D, int buf) {
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  const ProbState& s = D.st[pi];
  int ld;
  const float2* X = buf_base(D, buf, p, ld);
  unsigned long long* am = (unsigned long long*)(D.small + p.soff + D.L.argmx);
  if (s.done) return;
  const int w = min(s.wv, p.m);                 // argmx holds LDM >= m entries
  for (int j = 0; j < w; ++j) {
    unsigned long long best = 0ull;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p.N; r += gridDim.x * blockDim.x) {
      float2 v = X[(long long)j * ld + r];
      float a2 = v.x * v.x + v.y * v.y;
      unsigned long long key = ((unsigned long long)__float_as_uint(a2) << 32) | (0xFFFFFFFFull - (unsigned)r);
      best = key > best ? key : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long oth = __shfl_xor_sync(0xffffffffu, best, o);
      best = oth > best ? oth : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&am[j], best);
  }
}

// ----------------------------------------------------------------------------- Vandermonde RHS / residual
// rhs: b_i = sum_{k in I_n} conj(z_i^k) f(k);  resid: ||sum_j c_j z_j^k - f(k)||^2, all in FP64
// (the normal equations square the condition of A: nodes closer than 1/n, as in the Section 5
// workloads, need b to full FP64 accuracy).  z_i^k = prod_l E_l[i][k_l] with E_l[i][x] =
// exp(-+2 pi i t_i(l) x) from an FP64 recurrence, built once per block of RHS_ROWS rows.  For b,
// the threads split into m groups (one term each) that share the block's rows; for the
// residual each thread takes rows.
constexpr int RHS_ROWS = 1024;
constexpr int RHS_TABLE_MAX = 6144;          // d m (n + 1) (checked when a problem is accepted)

__global__ void __launch_bounds__(256) k_rhs(Dev D, int resid) {
  extern __shared__ double2 tab[];   // [d][m][n+1] powers, then [d][RHS_ROWS] digits (16-bit)
  __shared__ double2 part[256];
  __shared__ double shr[32];
  const int pi = blockIdx.y;
  const ProbDesc& p = D.P[pi];
  ProbState& s = D.st[pi];
  const int m = s.rank_used;
  if (s.done || m <= 0 || m > p.m) return;
  const int r0 = blockIdx.x * RHS_ROWS;
  if (r0 >= p.N) return;
  const int nrows = min(RHS_ROWS, p.N - r0);
  const int n1 = p.n + 1;
  short* kd = (short*)(tab + RHS_TABLE_MAX);       // kd[l * RHS_ROWS + rr]: digit l of row rr (n < 6144)
  const double* t = (const double*)(D.small + p.soff + D.L.t);
  const double2* c = (const double2*)(D.small + p.soff + D.L.c);
  const double sign = resid ? -1.0 : 1.0;
  const double2* zr = (const double2*)(D.small + p.soff + D.L.zraw);
  for (int q = threadIdx.x; q < p.d * m; q += blockDim.x) {
    int l = q / m, i = q % m;
    double2 e1;
    if (D.vand) {
      // raw eigenvalue z~ (Section 4 reading): conj(z) for the right-hand side, z for the model
      const double2 z = zr[i * PRONY_DMAX + l];
      e1 = make_double2(z.x, -sign * z.y);
    } else {
      double sn, cs;
      sincospi(2.0 * t[i * PRONY_DMAX + l], &sn, &cs);
      e1 = make_double2(cs, sign * sn);
    }
    double2 e = make_double2(1.0, 0.0);
    double2* row = tab + ((size_t)l * m + i) * n1;
    for (int x = 0; x < n1; ++x) {
      row[x] = e;
      e = cmul(e, e1);
    }
  }
  for (int rr = threadIdx.x; rr < nrows; rr += blockDim.x) {
    int rem = r0 + rr;
    for (int l = p.d - 1; l >= 0; --l) {
      kd[l * RHS_ROWS + rr] = (short)(rem % n1);
      rem /= n1;
    }
  }
  __syncthreads();
  auto power = [&](int i, int rr) {
    double2 e = tab[(size_t)i * n1 + kd[rr]];
    for (int l = 1; l < p.d; ++l) e = cmul(e, tab[((size_t)l * m + i) * n1 + kd[l * RHS_ROWS + rr]]);
    return e;
  };
  auto sample = [&](int rr) {
    int gi = 0, mul = 1;
    for (int l = p.d - 1; l >= 0; --l) {
      gi += (kd[l * RHS_ROWS + rr] + p.n) * mul;
      mul *= p.G;
    }
    return D.grid64[p.grid + gi];
  };
  if (!resid) {
    const int tpi = blockDim.x / m;                 // threads per term (m <= 64: at least 4)
    const int i = threadIdx.x / tpi, q = threadIdx.x % tpi;
    // four interleaved partial sums (FP64 additions have a long dependent latency), fixed order
    double2 a4[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    if (i < m) {
      int u = 0;
      for (int rr = q; rr < nrows; rr += tpi, u = (u + 1) & 3) a4[u] = cadd(a4[u], cmul(power(i, rr), sample(rr)));
    }
    part[threadIdx.x] = cadd(cadd(a4[0], a4[1]), cadd(a4[2], a4[3]));
    __syncthreads();
    double2* b = (double2*)(D.small + p.soff + D.L.rhs);
    double2* slots = (double2*)red_region(D, pi);
    if (i < m && q == 0 && ws_ok(D, 16LL * m * (blockIdx.x + 1) <= D.red_stride, 14)) {
      double2 sum = make_double2(0.0, 0.0);
      for (int u = 0; u < tpi; ++u) sum = cadd(sum, part[threadIdx.x + u]);
      slots[(size_t)blockIdx.x * m + i] = sum;
    }
    // block sums of b in block order
    const int nblk = (p.N + RHS_ROWS - 1) / RHS_ROWS;
    if (red_arrive(D, pi, nblk))
      for (int ii = threadIdx.x; ii < m; ii += blockDim.x) {
        double2 sum = b[ii];
        for (int k = 0; k < nblk; ++k) sum = cadd(sum, __ldcg(slots + (size_t)k * m + ii));
        b[ii] = sum;
      }
  } else {
    double r2 = 0.0;
    for (int rr = threadIdx.x; rr < nrows; rr += blockDim.x) {
      const double2 f = sample(rr);
      double2 v[2] = {make_double2(-f.x, -f.y), make_double2(0.0, 0.0)};   // two chains over the terms
      for (int i = 0; i < m; ++i) v[i & 1] = cadd(v[i & 1], cmul(c[i], power(i, rr)));
      r2 += cabs2(cadd(v[0], v[1]));
    }
    double tot = block_sum(r2, shr);
    double* slot = (double*)red_region(D, pi);
    if (threadIdx.x == 0 && ws_ok(D, 8LL * (blockIdx.x + 1) <= D.red_stride, 15)) slot[blockIdx.x] = tot;
    const int nblk = (p.N + RHS_ROWS - 1) / RHS_ROWS;
    if (red_arrive(D, pi, nblk) && threadIdx.x == 0) {
      double sum = 0.0;
      for (int k = 0; k < nblk; ++k) sum += __ldcg(slot + k);
      s.ls_num2 = sum;
    }
  }
}

// Packed outputs: t_out[(ooff + j) d + l], c_out[ooff + j]; entries past rank_used are zero.
__global__ void k_gather_out(Dev D, double* t_out, double2* c_out) {
  const int pi = blockIdx.x;
  const ProbDesc& p = D.P[pi];
  const ProbState& s = D.st[pi];
  const double* t = (const double*)(D.small + p.soff + D.L.t);
  const double2* c = (const double2*)(D.small + p.soff + D.L.c);
  for (int q = threadIdx.x; q < p.m * p.d; q += blockDim.x) {
    int j = q / p.d, l = q % p.d;
    t_out[(p.ooff + j) * D.maxD + l] = j < s.rank_used ? t[j * PRONY_DMAX + l] : 0.0;
  }
  for (int j = threadIdx.x; j < p.m; j += blockDim.x)
    c_out[p.ooff + j] = j < s.rank_used ? c[j] : make_double2(0.0, 0.0);
}

__global__ void k_copy_cols(Dev D, int buf, int wsel, double2* out) {
  const ProbDesc& p = D.P[0];
  const ProbState& s = D.st[0];
  int ld;
  const float2* X = buf_base(D, buf, p, ld);
  const int w = width_of(s, p, wsel);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)p.N * p.m;
       q += (long long)gridDim.x * blockDim.x) {
    int col = (int)(q / p.N), r = (int)(q % p.N);
    float2 v = col < w ? X[(long long)col * ld + r] : make_float2(0.f, 0.f);
    out[q] = make_double2(v.x, v.y);
  }
}

// ----------------------------------------------------------------------------- exponential sum (Eq. 1)
__global__ void __launch_bounds__(256) k_expsum_fwd(const double* t, const float2* c, int m, int d, Box B,
                                                    long long K, float2* f) {
  __shared__ uint64_t T[PRONY_MMAX * PRONY_DMAX];
  __shared__ float2 cs[PRONY_MMAX];
  for (int q = threadIdx.x; q < m * d; q += blockDim.x) T[q] = frac64(t[q]);
  for (int q = threadIdx.x; q < m; q += blockDim.x) cs[q] = c[q];
  __syncthreads();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < K; q += (long long)gridDim.x * blockDim.x) {
    int k[PRONY_DMAX];
    box_point(B, d, q, k);
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < m; ++j) {
      float u = centred_phase(T + j * d, k, d), sn, cn;
      sincospif(2.0f * u, &sn, &cn);                  // e = cn - i sn
      float2 cj = cs[j];
      acc.x += cj.x * cn + cj.y * sn;
      acc.y += cj.y * cn - cj.x * sn;
    }
    f[q] = acc;
  }
}

// acc[j][0..1] += sum_k g_k conj(e_jk);  acc[j][2+l] += sum_k k_l Im(conj(g_k) c_j e_jk)
__global__ void __launch_bounds__(256) k_expsum_bwd(const double* t, const float2* c, int m, int d, Box B,
                                                    long long K, const float2* g, double* acc) {
  __shared__ uint64_t T[PRONY_MMAX * PRONY_DMAX];
  __shared__ float2 cs[PRONY_MMAX];
  __shared__ float blk[PRONY_MMAX * (2 + PRONY_DMAX)];
  const int W = 2 + d;
  for (int q = threadIdx.x; q < m * d; q += blockDim.x) T[q] = frac64(t[q]);
  for (int q = threadIdx.x; q < m; q += blockDim.x) cs[q] = c[q];
  for (int q = threadIdx.x; q < m * W; q += blockDim.x) blk[q] = 0.f;
  __syncthreads();
  for (long long base = blockIdx.x * (long long)blockDim.x; base < K; base += (long long)gridDim.x * blockDim.x) {
    long long q = base + threadIdx.x;
    int k[PRONY_DMAX] = {0, 0, 0, 0};
    float2 gk = make_float2(0.f, 0.f);
    if (q < K) {
      box_point(B, d, q, k);
      gk = g[q];
    }
    for (int j = 0; j < m; ++j) {
      float u = centred_phase(T + j * d, k, d), sn, cn;
      sincospif(2.0f * u, &sn, &cn);
      float2 e = make_float2(cn, -sn);
      float gcx = gk.x * e.x + gk.y * e.y;            // g conj(e)
      float gcy = gk.y * e.x - gk.x * e.y;
      float2 ce = make_float2(cs[j].x * e.x - cs[j].y * e.y, cs[j].x * e.y + cs[j].y * e.x);
      float im = gk.x * ce.y - gk.y * ce.x;           // Im(conj(g) c e)
      float v[2 + PRONY_DMAX] = {gcx, gcy, im * k[0], im * k[1], im * k[2], im * k[3]};
#pragma unroll
      for (int w = 0; w < 2 + PRONY_DMAX; ++w) {
        if (w >= W) break;
        float x = v[w];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&blk[j * W + w], x);
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < m * W; q += blockDim.x) atomicAdd(&acc[q], (double)blk[q]);
}

__global__ void k_expsum_bwd_finish(const double* acc, int m, int d, double* gt, float2* gc) {
  const int W = 2 + d;
  const double two_pi = 6.283185307179586;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    gc[j] = make_float2((float)acc[j * W], (float)acc[j * W + 1]);
    for (int l = 0; l < d; ++l) gt[j * d + l] = two_pi * acc[j * W + 2 + l];
  }
}

__global__ void k_eval_points(const double* t, const double2* c, int m, int d, const int* k, int K, double2* f) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < K; q += gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < m; ++j) {
      uint64_t a = 0;
      for (int l = 0; l < d; ++l) a += frac64(t[j * d + l]) * (uint64_t)(long long)k[(long long)q * d + l];
      double u = (double)(long long)a * 5.421010862427522e-20;   // 2^-64
      double sn, cn;
      sincospi(2.0 * u, &sn, &cn);
      acc = cadd(acc, cmul(c[j], make_double2(cn, -sn)));
    }
    f[q] = acc;
  }
}

inline int blocks_for(long long n, int per) { return (int)std::min<long long>((n + per - 1) / per, 1 << 16); }

}  // namespace

#include <algorithm>

void launch_prep(const Dev& D, cudaStream_t s) {
  note_launch();
  k_state_init<<<(D.nprob + 127) / 128, 128, 0, s>>>(D);
  dim3 g(blocks_per_problem(std::min((D.maxGd + 255) / 256, 64), D.nprob), D.nprob);
  note_launch();
  k_prep<<<g, 256, 0, s>>>(D);
}

void launch_init_v0(const Dev& D, unsigned long long seed, cudaStream_t s) {
  dim3 g(blocks_per_problem(std::min((D.maxN + 255) / 256, 256), D.nprob), D.nprob);
  note_launch();
  k_init_v0<<<g, 256, 0, s>>>(D, seed);
}

void launch_zero_small(const Dev& D, long long off, long long bytes, cudaStream_t s) {
  dim3 g(blocks_per_problem(std::min<long long>((bytes / 4 + 255) / 256, 32), D.nprob), D.nprob);
  note_launch();
  k_zero_small<<<g, 256, 0, s>>>(D, off, bytes);
}

// The dynamic shared memory attribute of k_gram only ever grows (a launch needs it to cover its
// own size; lowering it for a smaller batch would make a later larger launch fail).
static size_t g_gram_attr = 0;
static void gram_attr(size_t sm) {
  if (sm > g_gram_attr) {
    cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    g_gram_attr = sm;
  }
}

// Launch geometry of k_gram for a batch: dynamic shared memory, rows per block and blocks per
// problem (the batch fills the resident blocks once, at least RS rows per block).
static void gram_geometry(const Dev& D, size_t& sm, int& chunk, int& nblk) {
  static std::map<size_t, int> slots_for;      // shared memory size -> resident blocks on the GPU
  // two buffers of staged rows of X and Z (float4 per value); afterwards the same space holds the
  // row-group partial sums, (RG - 1) x tiles x 16 packed entries with RG = min(RS, 256 / tiles):
  // fewer than 256 x 16
  const int RS = gram_rows(D.L.LDR);
  sm = std::max(sizeof(float4) * (4 * (size_t)D.L.LDR * (RS + 1)), sizeof(unsigned long long) * 256 * 16);
  auto it = slots_for.find(sm);
  if (it == slots_for.end()) {
    int occ = 1, dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    gram_attr(sm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram, 256, sm) != cudaSuccess) {
      cudaGetLastError();
      occ = 2;
    }
    it = slots_for.emplace(sm, std::max(1, occ) * sms).first;
  }
  // at most 64 blocks per problem: the last block of a problem adds every block's partial Gram
  const int per_prob = std::max(1, std::min(64, it->second / std::max(1, D.nprob)));
  chunk = std::max(RS, (D.maxN + per_prob - 1) / per_prob);
  chunk = (chunk + RS - 1) / RS * RS;
  nblk = (D.maxN + chunk - 1) / chunk;
}

long long red_bytes_per_problem(const Dev& D) {
  size_t sm;
  int chunk, nblk;
  gram_geometry(D, sm, chunk, nblk);
  long long b = (long long)nblk * D.L.LDR * D.L.LDR * (long long)sizeof(float2);           // k_gram
  b = std::max<long long>(b, 64LL * sizeof(double2));                                         // k_prep (<= 64 blocks)
  b = std::max<long long>(b, (D.maxN + 63) / 64 * (long long)sizeof(double));                // k_apply norms
  b = std::max<long long>(b, (D.maxN + RHS_ROWS - 1) / RHS_ROWS * (long long)std::max(1, D.L.LDM) *
                                 (long long)sizeof(double2));                                  // k_rhs
  return (b + 255) / 256 * 256;
}

void launch_gram(const Dev& D, int xbuf, int xshift, int xw, int zbuf, int zshift, int zw, long long out_off,
                 int out_ld, cudaStream_t s) {
  size_t sm;
  int chunk, nblk;
  gram_geometry(D, sm, chunk, nblk);
  gram_attr(sm);
  dim3 g(nblk, D.nprob);
  note_launch();
  k_gram<<<g, 256, sm, s>>>(D, xbuf, xshift, xw, zbuf, zshift, zw, out_off, out_ld, chunk);
}

void launch_apply(const Dev& D, int xbuf, int xw, int outw, long long m_off, int m_double, int zbuf, int outbuf,
                  int norm_only, cudaStream_t s) {
  static size_t set = 0;
  const int rows = D.L.LDR <= 64 ? 128 : 64;
  const size_t sm = sizeof(float2) * ((size_t)D.L.LDR * ((D.L.LDR + 3) & ~3) + (size_t)D.L.LDR * rows);
  if (sm > set) {
    cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set = sm;
  }
  dim3 g((D.maxN + rows - 1) / rows, D.nprob);
  note_launch();
  k_apply<<<g, 256, sm, s>>>(D, xbuf, xw, outw, m_off, m_double, zbuf, outbuf, norm_only, rows);
}

void launch_argmax(const Dev& D, int buf, cudaStream_t s) {
  dim3 g(std::max(1, std::min((D.maxN + 255) / 256, 64)), D.nprob);
  note_launch();
  k_argmax<<<g, 256, 0, s>>>(D, buf);
}

void launch_rhs(const Dev& D, int resid, cudaStream_t s) {
  static bool attr = false;
  const size_t sm = sizeof(double2) * RHS_TABLE_MAX + sizeof(short) * PRONY_DMAX * RHS_ROWS;
  if (!attr) {
    cudaFuncSetAttribute(k_rhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 g((D.maxN + RHS_ROWS - 1) / RHS_ROWS, D.nprob);
  note_launch();
  k_rhs<<<g, 256, sm, s>>>(D, resid);
}

void launch_gather_out(const Dev& D, double* t_out, double2* c_out, cudaStream_t s) {
  note_launch();
  k_gather_out<<<D.nprob, 128, 0, s>>>(D, t_out, c_out);
}

void launch_copy_cols(const Dev& D, int buf, int w_sel, double2* out, cudaStream_t s) {
  note_launch();
  k_copy_cols<<<64, 256, 0, s>>>(D, buf, w_sel, out);
}

void launch_expsum_fwd(const double* t, const float2* c, int m, int d, const int* lo, const int* len, long long K,
                       float2* f, cudaStream_t s) {
  note_launch();
  k_expsum_fwd<<<blocks_for(K, 256), 256, 0, s>>>(t, c, m, d, make_box(d, lo, len), K, f);
}

void launch_expsum_bwd(const double* t, const float2* c, int m, int d, const int* lo, const int* len, long long K,
                       const float2* g, double* acc, cudaStream_t s) {
  int nb = std::min(blocks_for(K, 256), 4 * 152);
  note_launch();
  k_expsum_bwd<<<nb, 256, 0, s>>>(t, c, m, d, make_box(d, lo, len), K, g, acc);
}

void launch_expsum_bwd_finish(const double* acc, int m, int d, double* gt, float2* gc, cudaStream_t s) {
  note_launch();
  k_expsum_bwd_finish<<<1, 64, 0, s>>>(acc, m, d, gt, gc);
}

void launch_eval_points(const double* t, const double2* c, int m, int d, const int* k, int K, double2* f,
                        cudaStream_t s) {
  note_launch();
  k_eval_points<<<blocks_for(K, 128), 128, 0, s>>>(t, c, m, d, k, K, f);
}
