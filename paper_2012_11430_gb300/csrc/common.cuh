// Shared definitions of the Prony CUDA library (device side and launchers).
//
// Layout in HBM (one workspace per context, grown on demand; all problems of a
// batch side by side, offsets in ProbDesc):
//   grid64  complex128 samples of every problem, (2n+2)^d each (input copy)
//   gF, gH  complex64 copies of F(x) = f(x) and F(x) = conj f(-x) on the same
//           grid (the Toeplitz functions of T and T^*), (2n+2)^d each
//   V, U, B1, B2   N x r0 complex64, column-major, leading dimension N
//   Y       (n+2)^d x r0 complex64 column-major: rows of T V over the box
//           {0..n+1}^d, which holds T V (rows k in I_n) and every T_l V
//           (rows k + e_l) of Eq. generateSl at once
//   small   per-problem FP64 / FP32 workspace for the r0 x r0 and m x m steps
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// per-problem status codes (the values of prony_status in the public header)
#define ST_OK 0
#define ST_ERANK (-2)
#define ST_ENOCONV (-3)
#define ST_ENAN (-4)

#define PRONY_RMAX 128        // max columns r0 = m + p
#define PRONY_LM_PMAX 160     // max real parameters m (d + 2) of the refinement
#define PRONY_MMAX 64         // max terms m
#define PRONY_DMAX 4          // max dimension d

struct ProbDesc {
  int d, n, m, r0;            // dimension, grid size, terms, power-method width
  int N, Next, G, Gd;         // (n+1)^d, (n+2)^d, 2n+2, (2n+2)^d
  long long grid;             // offset (elements) of the problem's grid in grid64 / gF / gH
  long long xoff;             // offset (elements) of its N x r0 blocks in the X buffers
  long long yoff;             // offset (elements) of its Next x r0 block in Y
  long long soff;             // offset (bytes) of its small workspace
  long long ooff;             // offset (terms) of its results in the packed t / c outputs
  long long toff;             // offset (words) of its split-plane tables in tabF / tabH
  int Gd4;                    // Gd rounded up to a multiple of 4 (length of one table)
  int fL;                     // FFT products: points per axis of the circulant embedding (0: dense)
  long long foff;             // FFT products: offset (elements) of the problem's transform in fhat
};

// Per-problem iteration state, device resident.
struct ProbState {
  int wu, wv;                 // current widths of U and V
  int w_in, w_out;            // widths of the pending X -> X M product (set by the Cholesky step)
  int iter;                   // power iterations done
  int done;                   // 1: stopped, later iterations skip this problem
  int status;                 // prony_status
  int rank_det;               // detected rank (pivoted QR of the first T^* U)
  int rank_used;
  int nonfinite;
  double normT2;              // ||T||_F^2 (closed form)
  double normf2;              // ||f||_2^2 over I_n
  double resid2;              // ||R_k||_F^2
  double resid2_prev;
  double ls_num2;             // ||A^T c - f||^2
  double sigma_ratio;
  int lk;                     // Lanczos (Algorithm 2): vectors u_1..u_lk accepted
  int lstop;                  // Lanczos: why it stopped (1 alpha, 2 beta below the tolerance, 3 block full)
  double lalpha, lbeta;       // Lanczos: last alpha, beta
  int oa_conv;                // refinement of the SVD of Q: 0 running, 2 last step pending, 1 converged
};

// Small per-problem workspace: byte offsets inside the block at ProbDesc::soff.
// LDR >= every r0 of the batch, LDM >= every m (leading dimensions of the blocks).
struct SmallLay {
  int LDR, LDM;
  long long gram;    // LDR x LDR double2  Gram of a tall block
  long long mapm;    // LDR x LDR float2   P R^{-1} of the last Cholesky step
  long long q;       // LDR x LDM double2  Q = U^* T V
  long long mproj;   // d x LDR x LDM double2  U^* T_l V
  long long uq;      // LDR x LDM double2  left singular vectors of Q
  long long vq;      // LDM x LDM double2  right singular vectors of Q
  long long sigma;   // LDM double
  long long S;       // d x LDM x LDM double2
  long long t;       // LDM x DMAX double
  long long rhs;     // LDM double2
  long long c;       // LDM double2
  long long phase;   // LDM double2
  long long argmx;   // LDM u64
  long long work1, work2, work3, work4;   // LDR x LDM double2 scratch of the FP64 steps
  long long zraw;    // LDM x DMAX double2  eigenvalues z_j(l) of the S_l
  long long bytes;
};

inline SmallLay make_small_lay(int LDR, int LDM, int dmax) {
  SmallLay L;
  L.LDR = LDR;
  L.LDM = LDM;
  long long o = 0;
  auto take = [&](long long b) { long long r = o; o += (b + 15) / 16 * 16; return r; };
  L.gram = take(16LL * LDR * LDR);
  L.mapm = take(8LL * LDR * LDR);
  L.q = take(16LL * LDR * LDM);
  L.mproj = take(16LL * dmax * LDR * LDM);
  L.uq = take(16LL * LDR * LDM);
  L.vq = take(16LL * LDM * LDM);
  L.sigma = take(8LL * LDM);
  L.S = take(16LL * dmax * LDM * LDM);
  L.t = take(8LL * LDM * PRONY_DMAX);
  L.rhs = take(16LL * LDM);
  L.c = take(16LL * LDM);
  L.phase = take(16LL * LDM);
  L.argmx = take(8LL * LDM);
  L.work1 = take(16LL * LDR * LDM);
  L.work2 = take(16LL * LDR * LDM);
  L.work3 = take(16LL * LDR * LDM);
  L.work4 = take(16LL * LDR * LDM);
  L.zraw = take(16LL * LDM * PRONY_DMAX);
  L.bytes = (o + 255) / 256 * 256;
  return L;
}

// Every device pointer a kernel may need, passed by value.
struct Dev {
  const ProbDesc* P;
  ProbState* st;
  int nprob;
  int maxN, maxNext, maxGd, maxR0, maxM, maxD;
  const double2* grid64;
  float2* gF;
  float2* gH;
  // Split BF16 planes of the samples for the tensor-core path (Section 1 samples, split once):
  // table a = part * 3 + plane (part 0: Re, 1: Im) of problem p at toff + a * Gd4; word x holds
  // plane(F[x]) in its low half and plane(F[x - 1]) in its high half (F = gF for tabF, gH for tabH).
  uint32_t* tabF;
  uint32_t* tabH;
  float2* V;
  float2* U;
  float2* B1;
  float2* B2;
  float2* Y;
  char* small;
  SmallLay L;
  int vand;          // least-squares matrix from t (0) or from the raw z (1)
  // FFT products: transforms of the embedded samples (scrambled order) and exp(-2 pi i j / fLT)
  float2* fhat;
  float2* ftw;
  int fLT;
  // iteration caps of the small FP32 iterations (0: defaults, 30 Jacobi sweeps and 30 m + 30
  // shifted-QR steps); lowered only to exercise the PRONY_ENOCONV path
  int cap_jacobi, cap_eigqr;
  // fixed-order sums over the blocks of one problem: `red_stride` bytes of partials per problem,
  // one arrival counter per problem (zero between launches)
  char* red;
  long long red_stride;
  int* rcnt;
  // first failed workspace bound check (site number, 0: none); the host turns it into PRONY_ECUDA
  int* oob;
};

// Bound check of a workspace access: on failure records `site` in D.oob (first failure wins)
// and returns false, so that the caller skips the access instead of writing out of bounds.
__device__ inline bool ws_ok(const Dev& D, bool ok, int site) {
  if (!ok && D.oob) atomicCAS(D.oob, 0, site);
  return ok;
}

// Deterministic cross-block sums: every block of problem `pi` that takes part stores its
// partial values in its own slot of the problem's region of D.red, then calls red_arrive with
// the number of blocks taking part.  It returns true in every thread of the last block to arrive
// (all other partials are then visible to it), which adds the slots in block order -- so the
// result does not depend on the order in which the blocks finish.  The counter is reset for the
// next launch.  Every thread of the block must call it.
__device__ inline bool red_arrive(const Dev& D, int pi, int expected) {
  __shared__ int s_last_block;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int old = atomicAdd(&D.rcnt[pi], 1);
    s_last_block = old == expected - 1;
    if (s_last_block) D.rcnt[pi] = 0;
  }
  __syncthreads();
  const bool last = s_last_block != 0;
  if (last) __threadfence();
  return last;
}
__device__ inline char* red_region(const Dev& D, int pi) { return D.red + (size_t)pi * D.red_stride; }

// ----------------------------------------------------------------------------- complex helpers
__host__ __device__ inline float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline double cabsd(double2 a) { return hypot(a.x, a.y); }
__device__ inline double2 cdiv(double2 a, double2 b) {  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  double r = b.x / b.y, den = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ inline double2 csqrtd(double2 a) {
  double r = hypot(a.x, a.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  double sx = sqrt(0.5 * (r + fabs(a.x)));
  if (a.x >= 0.0) return make_double2(sx, a.y / (2.0 * sx));
  return make_double2(fabs(a.y) / (2.0 * sx), a.y >= 0.0 ? sx : -sx);
}

// ----------------------------------------------------------------------------- index maps
// Row r of I_n (row-major, (n+1)^d rows) -> row of the box {0..L-1}^d after adding
// the unit vector e_shift (shift < 0: none).
__device__ inline int map_row(int r, int n, int d, int L, int shift) {
  int idx = 0, mul = 1, rem = r;
  for (int l = d - 1; l >= 0; --l) {
    int k = rem % (n + 1);
    rem /= (n + 1);
    if (l == shift) k += 1;
    idx += k * mul;
    mul *= L;
  }
  return idx;
}

// ----------------------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw (SC'11).  Draw convention: key = (seed, stream),
// counter = (index, 0, 0, 0); u = ((w >> 11) + 0.5) 2^-53; complex normal
// z = sqrt(-log u0) exp(2 pi i u1).
#define PRONY_STREAM_MU 0x4D55ull
#define PRONY_STREAM_V0 0x5630ull
__host__ __device__ inline void philox4x64(uint64_t ctr[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    uint64_t hi0 = __umul64hi(M0, ctr[0]), lo0 = M0 * ctr[0];
    uint64_t hi1 = __umul64hi(M1, ctr[2]), lo1 = M1 * ctr[2];
#else
    unsigned __int128 p0 = (unsigned __int128)M0 * ctr[0], p1 = (unsigned __int128)M1 * ctr[2];
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0, hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
#endif
    uint64_t c0 = hi1 ^ ctr[1] ^ k0, c2 = hi0 ^ ctr[3] ^ k1;
    ctr[0] = c0; ctr[1] = lo1; ctr[2] = c2; ctr[3] = lo0;
    k0 += W0; k1 += W1;
  }
}
__host__ __device__ inline double philox_u01(uint64_t w) { return ((double)(w >> 11) + 0.5) * 1.1102230246251565e-16; }

// t in [0,1) as a 64-bit binary fraction: <t, k> mod 1 is then exact integer arithmetic.
__device__ inline uint64_t frac64(double t) {
  double f = t - floor(t);
  // f * 2^64, split to keep all 53 bits
  uint64_t hi = (uint64_t)(f * 4294967296.0);
  double rem = f * 4294967296.0 - (double)hi;
  uint64_t lo = (uint64_t)(rem * 4294967296.0);
  return (hi << 32) + lo;
}

// Integer box {lo_l .. lo_l + len_l - 1} enumerated row-major (last coordinate fastest).
struct Box { int lo[PRONY_DMAX]; int len[PRONY_DMAX]; };

inline Box make_box(int d, const int* lo, const int* len) {
  Box B = {};
  for (int l = 0; l < d; ++l) { B.lo[l] = lo[l]; B.len[l] = len[l]; }
  return B;
}

__device__ inline void box_point(const Box& B, int d, long long q, int* k) {
  for (int l = d - 1; l >= 0; --l) {
    k[l] = B.lo[l] + (int)(q % B.len[l]);
    q /= B.len[l];
  }
}

// Phase <t_j, k> mod 1 from 64-bit binary fractions (exact), centred to [-1/2, 1/2).
__device__ inline float centred_phase(const uint64_t* T, const int* k, int d) {
  uint64_t acc = 0;
  for (int l = 0; l < d; ++l) acc += T[l] * (uint64_t)(long long)k[l];
  return (float)(int)(acc >> 32) * 2.3283064365386963e-10f;
}

// ----------------------------------------------------------------------------- launchers
// Every kernel launch of the library goes through a launcher that calls note_launch()
// (a process-wide counter, read with prony_get_stats).
void note_launch();
// Blocks per problem of a grid-stride kernel over every problem of a batch: `want` (sized for the
// largest problem), fewer for large batches, so that a launch holds at most ~16k blocks (with
// thousands of small problems, most blocks of a larger grid start, find no work and retire).
inline int blocks_per_problem(long long want, int nprob) {
  const long long cap = 16384LL / (nprob > 0 ? nprob : 1);
  const long long b = want < cap ? want : cap;
  return (int)(b > 1 ? b : 1);
}
// Message returned by prony_last_error() on this host thread.
void set_last_error(const char* msg);

// Column counts of the tall blocks, selected per problem: r0, the current U / V widths, m, the
// pending X -> X M product, a single column, and the Lanczos basis sizes k and k + 1.
enum WidthSel { W_R0 = 0, W_U = 1, W_V = 2, W_M = 3, W_IN = 4, W_OUT = 5, W_ONE = 6, W_LK = 7, W_LK1 = 8 };
__host__ __device__ inline int sel_width(const ProbState& s, const ProbDesc& p, int sel) {
  switch (sel) {
    case W_R0: return p.r0;
    case W_U: return s.wu;
    case W_V: return s.wv;
    case W_M: return p.m;
    case W_IN: return s.w_in;
    case W_OUT: return s.w_out;
    case W_ONE: return 1;
    case W_LK: return s.lk;
    default: return s.lk + 1;
  }
}
enum BufSel { BUF_V = 0, BUF_U = 1, BUF_B1 = 2, BUF_B2 = 3, BUF_Y = 4 };

// kernels_tall.cu
// Bytes of cross-block partials per problem that the tall kernels need for a batch of this
// layout (D.nprob, D.maxN, D.maxGd, D.L set).
long long red_bytes_per_problem(const Dev& D);
void launch_prep(const Dev& D, cudaStream_t s);
void launch_init_v0(const Dev& D, unsigned long long seed, cudaStream_t s);
void launch_zero_small(const Dev& D, long long off, long long bytes, cudaStream_t s);
// out[a][b] (+)= sum_{r in I_n} conj(X[map(r), a]) Z[map(r), b]; X, Z buffers with row shifts
void launch_gram(const Dev& D, int xbuf, int xshift, int xw, int zbuf, int zshift, int zw,
                 long long out_off, int out_ld, cudaStream_t s);
// OUT[r, j] = (zbuf >= 0 ? Z[r, j] : 0) - sum_a X[r, a] M[a][j] for r in I_n (without Z: + the sum); M in the small workspace
// (float2 at mapm, ld RMAX) or double2 (m_double, at m_off with ld MMAX).  norm_only: accumulate
// ||OUT||^2 into st.resid2 and do not store.
void launch_apply(const Dev& D, int xbuf, int xw, int outw, long long m_off, int m_double, int zbuf,
                  int outbuf, int norm_only, cudaStream_t s);
void launch_argmax(const Dev& D, int buf, cudaStream_t s);
void launch_rhs(const Dev& D, int resid, cudaStream_t s);
void launch_gather_out(const Dev& D, double* t_out, double2* c_out, cudaStream_t s);
void launch_copy_cols(const Dev& D, int buf, int w_sel, double2* out, cudaStream_t s);
void launch_expsum_fwd(const double* t, const float2* c, int m, int d, const int* lo, const int* len,
                       long long K, float2* f, cudaStream_t s);
void launch_expsum_bwd(const double* t, const float2* c, int m, int d, const int* lo, const int* len,
                       long long K, const float2* g, double* acc, cudaStream_t s);
void launch_expsum_bwd_finish(const double* acc, int m, int d, double* gt, float2* gc, cudaStream_t s);
void launch_eval_points(const double* t, const double2* c, int m, int d, const int* k, int K, double2* f,
                        cudaStream_t s);

// kernels_toeplitz.cu
// One CTA of a Toeplitz product: problem, row tile, K range ks of nks.  The K ranges of a row tile
// are consecutive jobs (ks innermost): with a K split the CTA of range 0 is job blockIdx - ks.
struct ToeplitzJob { int prob, mt, ks, nks; };
// Split K workspace: `part` holds one slot of simt_part_elems(maxw) complex64 per job, `cnt` one
// zeroed int per job (every launch leaves it zeroed).
size_t simt_part_elems(int maxw);
void launch_toeplitz(const Dev& D, const ToeplitzJob* jobs, int njobs, int adjoint, int xbuf, int wsel, int ybuf,
                     int y_ext, int maxw, float2* part, int* cnt, long long part_jobs, cudaStream_t s);

// kernels_tc.cu (tensor-core Toeplitz products: split BF16 planes or TF32 hi + lo)
// Window of a product CTA in its split-plane tables, [lo, lo + len) in table entries, for the grid
// indices [f_lo, f_hi] it reads.  TF32 tables hold one 32-bit entry per grid index x; BF16
// tables hold 16-bit entries in reverse order (entry Gd4 - 1 - x holds sample x), so that two
// consecutive input points on a grid line are two ascending entries (one 32-bit word, or two
// joined by a funnel shift).  Starts are 16-byte aligned; a BF16 window carries 8 spare entries
// (the word pairs of a line read up to two entries past its last point).
__host__ __device__ inline void tc_window(bool bf16, int Gd4, int f_lo, int f_hi, int& lo, int& len) {
  if (bf16) {
    const int r_lo = (Gd4 - 1 - f_hi) & ~7, r_hi = Gd4 - 1 - f_lo;
    lo = r_lo;
    len = ((r_hi - r_lo + 1 + 7) & ~7) + 8;
  } else {
    lo = f_lo & ~3;
    len = ((f_hi - lo + 1) + 3) & ~3;
  }
}
int tc_planes(int kind);
size_t tc_stage_bytes(int kind, int ntbox);
size_t tc_elem_bytes(int kind);
size_t tc_smem_bytes(int kind, int ntbox, int stages, int win_cap);
long long tc_prob_stride(int kind, int ntbox, int maxnc);
// Split K workspace of the tensor-core products: tc_part_floats(ntbox) floats per job, one zeroed
// counter per job.
size_t tc_part_floats(int ntbox);
void launch_split_tables(const Dev& D, int kind, cudaStream_t s);
void launch_xb_prep(const Dev& D, int xbuf, int xshift, int wsel, void* xb, int kind, long long prob_stride,
                    cudaStream_t s);
cudaError_t launch_toeplitz_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int adjoint, int wsel, int ybuf,
                               int y_ext, int kind, int ntbox, int win_cap, int stages, const void* xb,
                               long long prob_stride, float* part, int* cnt, long long part_jobs, int* err,
                               cudaStream_t s);
cudaError_t launch_gram_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int xbuf, int xshift, int xw, int zw,
                           long long out_off, int out_ld, int ntbox, int stages, const void* xb, long long prob_stride,
                           float* part, int* cnt, long long part_jobs, int* err, cudaStream_t s);
// OUT = X M (as launch_apply without Z and norm) on the tensor cores, three BF16 planes; jobs: one
// per row tile of the N rows, nks = 1; OUT is not the box buffer Y.
cudaError_t launch_apply_tc(const Dev& D, const ToeplitzJob* jobs, int njobs, int xbuf, int xw, int outw,
                            long long m_off, int m_double, int outbuf, int ntbox, int stages, void* xb,
                            long long prob_stride, int* err, cudaStream_t s);

// kernels_refine.cu (Levenberg-Marquardt refinement of (t, c))
long long lm_workspace_bytes(int m, int d);
size_t lm_solve_smem(int m, int d);
cudaError_t lm_set_attributes(int m, int d);
void launch_refine_lm(double* t, double2* c, int m, int d, const int* lo, const int* len, long long K,
                      const float2* y, int iters, double lambda0, double* hist, void* ws, cudaStream_t s);
constexpr int LM_LAUNCHES_PER_STEP = 4;

// kernels_lanczos.cu (Algorithm 2, batched)
// kernels_small.cu: condition node of the device-side power loop (CUDA graph WHILE node)
void launch_loop_cond(cudaGraphConditionalHandle h, const int* all_done, int* count, int cap, cudaStream_t s);

// kernels_fft.cu (Toeplitz products by circulant embedding and FP32 FFTs)
int fft_length(int n);
long long fft_points_host(int n, int d);   // points of one embedded grid in shared memory (padded)
void launch_fft_tables(const Dev& D, int maxpts, cudaStream_t s);
void launch_toeplitz_fft(const Dev& D, int maxpts, int maxw, int adjoint, int xbuf, int wsel, int ybuf, int y_ext,
                         cudaStream_t s);

void launch_lz_start(const Dev& D, cudaStream_t s);
void launch_lz_load(const Dev& D, int which, cudaStream_t s);
void launch_lz_axpy(const Dev& D, int which, cudaStream_t s);
void launch_lz_accept(const Dev& D, int which, double tol_rel, int cap, cudaStream_t s);
void launch_lz_finish(const Dev& D, cudaStream_t s);
void launch_lz_all_done(const Dev& D, int* flag, cudaStream_t s);

// kernels_small.cu
enum QrMode { QR_PLAIN = 0, QR_DROP = 1, QR_RANK = 2, QR_AUTO = 3 };   // AUTO: RANK on a problem's first iteration
void launch_chol(const Dev& D, int wsel, int target, int mode, double tol, int rank_mode, cudaStream_t s);
void launch_svd_S(const Dev& D, cudaStream_t s);
void launch_canon(const Dev& D, cudaStream_t s);
void launch_eig_t(const Dev& D, unsigned long long seed, cudaStream_t s);
void launch_solve_c(const Dev& D, cudaStream_t s);
void launch_check(const Dev& D, double tol_power, int max_iter, int* all_done, cudaStream_t s);
void launch_reset_done(const Dev& D, cudaStream_t s);
