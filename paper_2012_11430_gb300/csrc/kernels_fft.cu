// Toeplitz products by circulant embedding and FFTs (FP32), an alternative to the dense
// products for grids that fit one CTA's shared memory.
//
// T = [f(k - h)] with k in {0..n+1}^d (or I_n) and h in I_n = {0..n}^d only ever meets the
// differences k - h in {-n..n+1}^d, the sample grid of Section 1.  Embedded periodically in a
// grid of L >= 2n+2 points per axis (L a power of two), f becomes the kernel of an L^d circular
// convolution whose outputs at k coincide with (T x)_k: no difference wraps onto another one.
// So T x = IDFT(DFT(f_emb) * DFT(x_emb)) restricted to the rows, and T^* x uses conj(DFT(f_emb))
// (the embedding of conj f(-u) has the conjugate transform).
//
// The transforms are mixed-radix Cooley-Tukey in shared memory: the forward pass is a
// decimation in frequency that leaves its output in digit-reversed order, the inverse pass runs
// the same stages backwards from that order, so no reordering is ever done; DFT(f_emb) is stored
// in the same scrambled order by the same forward pass.  Each stage gives a thread R = 2..16
// points, transformed in registers by a radix-2 network with constant twiddles.  Pruning: the
// forward pass transforms only the lines that can hold nonzeros (x lives on {0..n}^d), and the
// inverse pass only the lines that reach the output rows.  Layout in shared memory: row-major
// over the axes with the last axis padded to P = L + 1 points (d >= 2), so that the threads of a
// warp, which take consecutive lines, hit distinct banks along every axis.
#include "common.cuh"

#include <algorithm>

namespace {

// exp(-2 pi i e / 16) for e = 0..7 (conjugated for the inverse)
constexpr float kC1 = 0.92387953251128674f;   // cos(pi/8)
constexpr float kS1 = 0.38268343236508978f;   // sin(pi/8)
constexpr float kH = 0.70710678118654752f;    // sqrt(1/2)

template <bool INV>
__device__ __forceinline__ float2 rot16(float2 t, int e) {
  float c, s;   // w = c - i s (forward)
  switch (e) {
    case 0: return t;
    case 4: return INV ? make_float2(-t.y, t.x) : make_float2(t.y, -t.x);
    case 1: c = kC1; s = kS1; break;
    case 2: c = kH; s = kH; break;
    case 3: c = kS1; s = kC1; break;
    case 5: c = -kS1; s = kC1; break;
    case 6: c = -kH; s = kH; break;
    default: c = -kC1; s = kS1; break;
  }
  if (INV) s = -s;
  return make_float2(t.x * c + t.y * s, t.y * c - t.x * s);
}

__host__ __device__ constexpr int bitrev(int k, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((k >> b) & 1) << (bits - 1 - b);
  return r;
}

template <int R>
struct Log2 { static constexpr int v = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4; };

// In-register DFT of R points by a radix-2 decimation-in-frequency network; the result of
// frequency k lands in x[bitrev(k)].
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&x)[R]) {
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int s0 = 0; s0 < R; s0 += 2 * span) {
#pragma unroll
      for (int i = 0; i < span; ++i) {
        const float2 a = x[s0 + i], b = x[s0 + i + span];
        x[s0 + i] = make_float2(a.x + b.x, a.y + b.y);
        x[s0 + i + span] = rot16<INV>(make_float2(a.x - b.x, a.y - b.y), i * (8 / span));
      }
    }
  }
}

// The line set of one axis: nl lines of L points at element stride es.  A line is fixed by its
// coordinates on the other axes (no = d - 1 of them, slowest first, extents ext, strides str):
// those before the transformed axis run below E (pruning), those after it over [0, L).
struct Lines {                                    // d <= 3 (checked when the batch is set up)
  int nl, es, no;
  int ext[2], str[2];
  __device__ int base(int li) const {
    if (no == 0) return 0;
    if (no == 1) return li * str[0];
    const int f = li % ext[1], sl = li / ext[1];
    return sl * str[0] + f * str[1];
  }
};

// stride of axis m in the padded layout
__device__ inline int axis_stride(int L, int P, int d, int m) {
  if (m == d - 1) return 1;
  int s = P;
  for (int l = m + 1; l < d - 1; ++l) s *= L;
  return s;
}

// Where a stage reads its points and where it writes its results.  The first stage of an axis
// (M = L) may take its points from the column in HBM (the last axis of the first forward pass)
// or treat the positions at and beyond `ein` along the axis as zero (they were never written:
// no zero fill is needed); the last forward stage may multiply by the spectrum of the samples
// (stored in the same scrambled order); the last inverse stage (M = L) may keep only the
// positions below `eout`, in shared memory or scaled into the output column in HBM.
enum { IN_SMEM = 0, IN_PRUNED = 1, IN_GLOBAL = 2 };
enum { OUT_SMEM = 0, OUT_SPECTRUM = 1, OUT_PRUNED = 2, OUT_GLOBAL = 3 };
struct StageIO {
  int in_mode, ein;
  const float2* X;      // column base, rows I_n (line li of the last axis starts at row li * ein)
  int out_mode, eout;
  const float2* F;      // spectrum (same layout as the shared array)
  int conjF;
  float2* Y;            // output column base (line li of the last axis starts at row li * eout)
  float scale;
};

// One stage (sub-blocks of M points, stride S = M / R) over every line of the set.
// L and M are powers of two (lgL, lgM their logarithms); tw holds exp(-2 pi i q / L), q < L, in
// shared memory.
template <int R, bool INV>
__device__ void fft_stage(float2* a, const Lines& ls, int lgL, int lgM, const float2* tw, const StageIO& io) {
  constexpr int B = Log2<R>::v;
  const int L = 1 << lgL, M = 1 << lgM;
  const int lgS = lgM - B, lgPL = lgL - B;
  const int items = ls.nl << lgPL;
  // consecutive threads take consecutive lines (distinct banks, see the layout) unless the stage
  // touches HBM, where consecutive points of a line keep the accesses coalesced
  const bool lines_fast = ls.no > 0 && io.in_mode != IN_GLOBAL && io.out_mode != OUT_GLOBAL;
  const int tws_lg = lgL - lgM;                    // twiddle w_M^e = tw[e << (lgL - lgM)]
  // (line, bj) of the first item and the step per blockDim.x items (lines fastest)
  int line = lines_fast ? (int)threadIdx.x % ls.nl : (int)threadIdx.x >> lgPL;
  int bj = lines_fast ? (int)threadIdx.x / ls.nl : (int)threadIdx.x & ((1 << lgPL) - 1);
  const int dl = lines_fast ? (int)blockDim.x % ls.nl : 0, dbj = lines_fast ? (int)blockDim.x / ls.nl : 0;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    if (!lines_fast) {
      line = it >> lgPL;
      bj = it & ((1 << lgPL) - 1);
    }
    const int b = bj >> lgS, j = bj & ((1 << lgS) - 1);
    const int S = 1 << lgS;
    float2* p = a + ls.base(line) + (b * M + j) * ls.es;
    const int step = S * ls.es;
    float2 x[R];
    if (io.in_mode == IN_GLOBAL) {              // M = L: the point of index q sits at position j + S q
      const float2* xl = io.X + (long long)line * io.ein;
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = j + S * q < io.ein ? xl[j + S * q] : make_float2(0.f, 0.f);
    } else if (io.in_mode == IN_PRUNED) {
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = j + S * q < io.ein ? p[q * step] : make_float2(0.f, 0.f);
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = p[q * step];
    }
    if (!INV) {
      dft_reg<R, false>(x);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        float2 y = x[bitrev(k, B)];
        if (k > 0 && j > 0) y = cmulf(y, tw[((j * k) & (M - 1)) << tws_lg]);
        if (io.out_mode == OUT_SPECTRUM) {
          const float2 f = __ldg(&io.F[(p - a) + k * step]);
          y = cmulf(y, io.conjF ? make_float2(f.x, -f.y) : f);
        }
        p[k * step] = y;
      }
    } else {
#pragma unroll
      for (int k = 1; k < R; ++k) {
        if (j > 0) {
          const float2 w = tw[((j * k) & (M - 1)) << tws_lg];
          x[k] = cmulf(x[k], make_float2(w.x, -w.y));
        }
      }
      dft_reg<R, true>(x);
      if (io.out_mode == OUT_GLOBAL) {          // M = L: output index q is position j + S q
        float2* yl = io.Y + (long long)line * io.eout;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const float2 v = x[bitrev(q, B)];
          if (j + S * q < io.eout) yl[j + S * q] = make_float2(v.x * io.scale, v.y * io.scale);
        }
      } else if (io.out_mode == OUT_PRUNED) {
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (j + S * q < io.eout) p[q * step] = x[bitrev(q, B)];
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) p[q * step] = x[bitrev(q, B)];
      }
    }
    if (lines_fast) {
      line += dl;
      bj += dbj;
      if (line >= ls.nl) {
        line -= ls.nl;
        ++bj;
      }
    }
  }
}

__device__ inline int stage_radix(int M) { return M >= 16 ? 16 : M; }

__device__ inline int ilog2(int v) { return 31 - __clz(v); }

template <bool INV>
__device__ void fft_stage_any(float2* a, const Lines& ls, int L, int M, const float2* tw, const StageIO& io) {
  const int lgL = ilog2(L), lgM = ilog2(M);
  switch (stage_radix(M)) {
    case 16: fft_stage<16, INV>(a, ls, lgL, lgM, tw, io); break;
    case 8: fft_stage<8, INV>(a, ls, lgL, lgM, tw, io); break;
    case 4: fft_stage<4, INV>(a, ls, lgL, lgM, tw, io); break;
    default: fft_stage<2, INV>(a, ls, lgL, lgM, tw, io); break;
  }
}

__device__ inline Lines axis_lines(int L, int P, int d, int axis, int E) {
  Lines ls;
  ls.es = axis_stride(L, P, d, axis);
  ls.no = 0;
  ls.nl = 1;
  for (int m = 0; m < d; ++m) {
    if (m == axis) continue;
    const int e = m < axis ? E : L;
    ls.ext[ls.no] = e;
    ls.str[ls.no] = axis_stride(L, P, d, m);
    ls.nl *= e;
    ++ls.no;
  }
  return ls;
}

// Forward transform of a fully populated grid (the samples' table), every line, last axis first.
__device__ void fft_forward_full(float2* a, int L, int P, int d, const float2* tw) {
  StageIO io{};
  for (int axis = d - 1; axis >= 0; --axis) {
    const Lines ls = axis_lines(L, P, d, axis, L);
    for (int M = L; M > 1; M /= stage_radix(M)) {
      fft_stage_any<false>(a, ls, L, M, tw, io);
      __syncthreads();
    }
  }
}

// Forward transform of the column x (nonzero on {0..n}^d, read from HBM), last axis first,
// ending with the product by the spectrum F (or its conjugate).  Lines whose coordinates on the
// axes not yet transformed exceed n are zero and skipped.
__device__ void fft_forward_column(float2* a, int L, int P, int d, int n, const float2* X, const float2* F,
                                   int conjF, const float2* tw) {
  for (int axis = d - 1; axis >= 0; --axis) {
    const Lines ls = axis_lines(L, P, d, axis, n + 1);
    for (int M = L; M > 1; M /= stage_radix(M)) {
      StageIO io{};
      if (M == L) {
        io.in_mode = axis == d - 1 ? IN_GLOBAL : IN_PRUNED;
        io.ein = n + 1;
        io.X = X;
      }
      if (axis == 0 && M == stage_radix(M)) {
        io.out_mode = OUT_SPECTRUM;
        io.F = F;
        io.conjF = conjF;
      }
      fft_stage_any<false>(a, ls, L, M, tw, io);
      __syncthreads();
    }
  }
}

// Inverse of the forward pass (scaled by 1/L^d), first axis first; only lines whose coordinates
// on the axes already back in the sample domain are below K are computed, and the last axis
// writes the rows of the box {0..K-1}^d straight into the output column Y.
__device__ void fft_inverse_column(float2* a, int L, int P, int d, int K, float2* Y, float scale, const float2* tw) {
  for (int axis = 0; axis < d; ++axis) {
    const Lines ls = axis_lines(L, P, d, axis, K);
    int Ms[16], ns = 0;
    for (int M = L; M > 1; M /= stage_radix(M)) Ms[ns++] = M;
    for (int s = ns - 1; s >= 0; --s) {
      StageIO io{};
      if (s == 0) {
        io.out_mode = axis == d - 1 ? OUT_GLOBAL : OUT_PRUNED;
        io.eout = K;
        io.Y = Y;
        io.scale = scale;
      }
      fft_stage_any<true>(a, ls, L, Ms[s], tw, io);
      __syncthreads();
    }
  }
}

__device__ inline int fft_pitch(const ProbDesc& p) { return p.d >= 2 ? p.fL + 1 : p.fL; }
__device__ inline int fft_points(const ProbDesc& p) {
  int v = fft_pitch(p);
  for (int l = 1; l < p.d; ++l) v *= p.fL;
  return v;
}

__global__ void k_fft_twiddles(float2* tw, int LT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= LT) return;
  double s, c;
  sincospi(2.0 * i / LT, &s, &c);
  tw[i] = make_float2((float)c, (float)-s);
}

// DFT of the embedded samples of every problem, in the scrambled order of fft_forward.
__global__ void __launch_bounds__(512) k_fft_table(Dev D) {
  extern __shared__ float2 a[];
  const ProbDesc& p = D.P[blockIdx.x];
  const int L = p.fL, d = p.d, P = fft_pitch(p), npts = fft_points(p);
  float2* tw = a + npts;                          // exp(-2 pi i q / L), q < L
  for (int q = threadIdx.x; q < L; q += blockDim.x) tw[q] = D.ftw[q * (D.fLT / L)];
  for (int i = threadIdx.x; i < npts; i += blockDim.x) a[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = threadIdx.x; i < p.Gd; i += blockDim.x) {
    int rem = i, g = 0;
    for (int l = d - 1; l >= 0; --l) {
      const int x = rem % p.G - p.n;          // coordinate in {-n..n+1}
      rem /= p.G;
      g += ((x + L) & (L - 1)) * axis_stride(L, P, d, l);
    }
    a[g] = D.gF[p.grid + i];
  }
  __syncthreads();
  fft_forward_full(a, L, P, d, tw);
  for (int i = threadIdx.x; i < npts; i += blockDim.x) D.fhat[p.foff + i] = a[i];
}

__device__ inline float2* fbuf(const Dev& D, int buf, const ProbDesc& p, int& ld) {
  switch (buf) {
    case BUF_V: ld = p.N; return D.V + p.xoff;
    case BUF_U: ld = p.N; return D.U + p.xoff;
    case BUF_B1: ld = p.N; return D.B1 + p.xoff;
    case BUF_B2: ld = p.N; return D.B2 + p.xoff;
    default: ld = p.Next; return D.Y + p.yoff;
  }
}

// One column of one problem per CTA: Y[:, col] = T X[:, col] (rows {0..n+1}^d when y_ext, else
// I_n) or T^* X[:, col] (adjoint, rows I_n).
__global__ void __launch_bounds__(512) k_toeplitz_fft(Dev D, int adjoint, int xbuf, int wsel, int ybuf, int y_ext) {
  extern __shared__ float2 a[];
  const ProbDesc& p = D.P[blockIdx.y];
  const ProbState& st = D.st[blockIdx.y];
  if (st.done) return;
  const int col = blockIdx.x;
  if (col >= sel_width(st, p, wsel)) return;
  const int L = p.fL, d = p.d, n = p.n, P = fft_pitch(p);
  int Ld = 1;
  for (int l = 0; l < d; ++l) Ld *= L;
  float2* tw = a + fft_points(p);                 // exp(-2 pi i q / L), q < L
  for (int q = threadIdx.x; q < L; q += blockDim.x) tw[q] = D.ftw[q * (D.fLT / L)];
  __syncthreads();
  int ldx = 0, ldy = 0;
  const float2* X = fbuf(D, xbuf, p, ldx);      // sets ldx: the offset is added afterwards
  float2* Y = fbuf(D, ybuf, p, ldy);
  X += (long long)col * ldx;
  Y += (long long)col * ldy;
  fft_forward_column(a, L, P, d, n, X, D.fhat + p.foff, adjoint, tw);
  fft_inverse_column(a, L, P, d, y_ext ? n + 2 : n + 1, Y, 1.0f / (float)Ld, tw);
}

int fft_threads(int maxpts) { return maxpts >= 8192 ? 512 : maxpts >= 2048 ? 256 : 128; }

}  // namespace

int fft_length(int n) {
  int L = 2;
  while (L < 2 * n + 2) L *= 2;
  return L;
}

long long fft_points_host(int n, int d) {
  const int L = fft_length(n);
  long long v = d >= 2 ? L + 1 : L;
  for (int l = 1; l < d; ++l) v *= L;
  return v;
}

void launch_fft_tables(const Dev& D, int maxpts, cudaStream_t s) {
  note_launch();
  k_fft_twiddles<<<(D.fLT + 255) / 256, 256, 0, s>>>(D.ftw, D.fLT);
  const size_t sm = sizeof(float2) * ((size_t)maxpts + D.fLT);
  cudaFuncSetAttribute(k_fft_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launch();
  k_fft_table<<<D.nprob, fft_threads(maxpts), sm, s>>>(D);
}

void launch_toeplitz_fft(const Dev& D, int maxpts, int maxw, int adjoint, int xbuf, int wsel, int ybuf, int y_ext,
                         cudaStream_t s) {
  const size_t sm = sizeof(float2) * ((size_t)maxpts + D.fLT);
  static size_t set = 0;
  if (sm > set) {
    cudaFuncSetAttribute(k_toeplitz_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set = sm;
  }
  note_launch();
  k_toeplitz_fft<<<dim3(maxw, D.nprob), fft_threads(maxpts), sm, s>>>(D, adjoint, xbuf, wsel, ybuf, y_ext);
}
