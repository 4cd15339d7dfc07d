// Host driver and C ABI of the Prony library (declarations in include/prony.h).
//
// One call runs Algorithm 1 for a batch of independent problems on one stream:
//   prep (grid copies, ||T||_F closed form) -> V_0 (Philox) -> CholeskyQR2(V_0)
//   -> Y = T V  [Toeplitz product over the box {0..n+1}^d]
//   -> loop (Algorithm 3):  U = qr(Y|I_n) ; Vbar = T^* U ; V = qr(Vbar) (column pivoting and
//      rank on the first pass) ; Y = T V ; Q = U^* Y|I_n ; ||Y|I_n - U Q||_F ; stop test
//   -> SVD(Q), S_l = U_Q^* (U^* Y_l) V_Q Sigma^{-1}  (Y_l = rows k + e_l of the last Y)
//   -> C_mu, eig, z, t -> conj(A) f, Gram, c -> ||A^T c - f||.
// Every kernel loops over the problems of the batch; problems that stopped skip work.
// The host waits once per power iteration to read the "all stopped" flag.
#include "common.cuh"
#include "../../include/prony.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#include <atomic>
#include <functional>

namespace {

thread_local std::string g_err;

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PRONY_ENOMEM : PRONY_ECUDA;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
};

int ensure(DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (b.cap >= bytes) return PRONY_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  b.cap = want;
  return PRONY_OK;
}

}  // namespace

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct prony_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  DBuf grid64, gF, gH, V, U, B1, B2, Y, small, P, st, jobs, flag, tout, cout, misc, misc2, misc3;
  DBuf xb, tabF, tabH, tcjobs, tcerr;   // tensor-core path: B' planes, split sample tables, jobs, error flag
  DBuf part, cnt;                       // split K products: partial tiles per job, arrival counters per tile
  DBuf red, rcnt;                       // fixed-order cross-block sums: partials and counters per problem
  DBuf oob;                             // first failed workspace bound check of a kernel (0: none)
  DBuf fhat, ftw;                       // FFT path: sample transforms, twiddles
  int* h_flag = nullptr;            // pinned
  std::vector<ProbState> h_st;
  // profiling of the Toeplitz launches
  bool prof = false;
  struct TRec { int ev; int iter; int ext; int wsel; };
  std::vector<TRec> trecs;
  std::vector<cudaEvent_t> events;  // pool, two per record
  std::vector<std::vector<ProbState>> snaps;
  prony_stats stats{};
  long long launch_base = 0;
  cudaError_t launch_err = cudaSuccess;   // first failed tensor-core launch of the current call
  std::map<std::string, int> tc_tuned;   // batch shape -> K split
  // the tensor-core job list on the device: (nks, P, then n and d of every problem) it was
  // built for, and its ext / in counts (a repeated batch layout skips the rebuild and the upload)
  std::vector<int> tcjob_sig;
  int tcjob_next = 0, tcjob_nin = 0, tcjob_ngram = 0, tcjob_napply = 0;
  // refinement: workspace and the CUDA graph of the last argument set
  DBuf lmws;
  struct LmKey {
    const void *t, *c, *y, *loss, *ws;
    int m, d, iters, lo[PRONY_DMAX], len[PRONY_DMAX];
    double lambda0;
  } lm_key{};
  cudaGraphExec_t lm_exec = nullptr;
  // the whole solve as one CUDA graph, for the last batch layout and options
  struct SolveGraph {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    long long fixed_launches = 0, body_launches[2] = {0, 0};
    bool has_loop[2] = {false, false};
  } solve_graph;
};

namespace {

struct HostProb {
  int d, n, m;
  long long sample_off, out_off;
};

double default_tol_power(int prec) {
  (void)prec;
  return 1e-6;
}

int validate(const HostProb& h) {
  if (h.d < 1 || h.d > PRONY_DMAX || h.n < 1 || h.m < 1 || h.m > PRONY_MMAX) return PRONY_EINVAL;
  double N = std::pow((double)(h.n + 1), h.d);
  if (N > 2.0e8 || h.m > N) return PRONY_EINVAL;
  if ((long long)h.d * h.m * (h.n + 1) > 6144) return PRONY_EINVAL;   // phase tables of the RHS kernel
  return PRONY_OK;
}

long long ipow(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Tensor-core configuration of a batch (split BF16 planes).
struct TcConf {
  bool on = false;
  bool tuned = false;                 // nks chosen (from the context's cache or by timing)
  int nks_min = 1;                    // tuning range: nks_min, 2 nks_min
  std::string key;                    // batch shape signature
  int kind = PRONY_BF16X3, ntbox = 16, stages = 2, win_cap = 0, nks = 1;
  long long prob_stride = 0;          // bytes of B' tiles per problem
  int njobs_ext = 0, njobs_in = 0;
  ToeplitzJob* jobs_ext = nullptr;
  ToeplitzJob* jobs_in = nullptr;
  int* err = nullptr;
  // tall-skinny Grams on the tensor cores (three BF16 planes): one CTA per problem and K range
  bool gram = false;
  int nks_gram = 1, gram_stages = 2, njobs_gram = 0;
  long long gram_stride = 0;          // bytes of the Gram's B' tiles per problem
  ToeplitzJob* jobs_gram = nullptr;
  // X M products of the tall blocks on the tensor cores (three BF16 planes): one CTA per row tile
  bool apply = false;
  int apply_stages = 2, njobs_apply = 0;
  long long apply_stride = 0;         // bytes of the B' tiles of M per problem
  ToeplitzJob* jobs_apply = nullptr;
};

struct Batch {
  std::vector<ProbDesc> P;
  Dev D{};
  int njobs_ext = 0, njobs_in = 0, nks = 1;
  ToeplitzJob* jobs_ext = nullptr;
  ToeplitzJob* jobs_in = nullptr;
  int maxw = 0;
  float2* part = nullptr;             // split K workspace of the products (FP32 path / tensor-core path)
  int* cnt = nullptr;
  long long part_jobs = 0;            // jobs the split K workspace holds
  TcConf tc;
  struct FftConf {
    bool on = false;  // every Toeplitz product by FFT (PRONY_FFT32)
    bool lz = false;  // the single-column products of the Lanczos steps only (other precisions)
    int maxpts = 0;   // largest embedded grid of the batch (shared memory of one CTA, in points)
  } fft;
};

// one embedded grid and its twiddles in shared memory: L = 128, d = 2 (padded) is 130 KB of complex64
constexpr int FFT_MAX_POINTS = 128 * 129 + 128;

bool is_tc(int prec) { return prec == PRONY_BF16X3 || prec == PRONY_BF16X2 || prec == PRONY_TF32X3; }

// host copies of the device index maps (window sizing)
int h_grid_of_row(int row, int L, const ProbDesc& p) {
  int g = 0, mul = 1, rem = row;
  for (int l = p.d - 1; l >= 0; --l) {
    g += (rem % L + p.n) * mul;
    rem /= L;
    mul *= p.G;
  }
  return g;
}
int h_grid_of_h(int h, const ProbDesc& p) {
  int g = 0, mul = 1, rem = h;
  for (int l = p.d - 1; l >= 0; --l) {
    g += (rem % (p.n + 1)) * mul;
    rem /= (p.n + 1);
    mul *= p.G;
  }
  return g;
}
// largest window (table entries, as the kernel sizes it: tc_window) over the CTAs of a problem
// for a K split into nks ranges
int max_window(const ProbDesc& p, int L, int nks, bool bf16) {
  const int rows = ipow(L, p.d) > 0 ? (int)ipow(L, p.d) : 0;
  const int nc = (p.N + 31) / 32, cper = (nc + nks - 1) / nks;
  int mx = 0;
  for (int r0 = 0; r0 < rows; r0 += 128) {
    int last = std::min(rows, r0 + 128) - 1;
    for (int ks = 0; ks < nks; ++ks) {
      int cb = ks * cper, ce = std::min(nc, cb + cper);
      if (cb >= ce) continue;
      int hf = 32 * cb, hl = std::min(p.N, 32 * ce) - 1;
      int lo = 0, len = 0;
      tc_window(bf16, p.Gd4, h_grid_of_row(r0, L, p) - h_grid_of_h(hl, p), h_grid_of_row(last, L, p) - h_grid_of_h(hf, p),
                lo, len);
      mx = std::max(mx, len);
    }
  }
  return mx;
}

// Split K workspace for `njobs` jobs of `slot_bytes` each: partial tiles and zeroed arrival
// counters (every product launch leaves its counters zeroed again).
int ensure_split_ws(prony_ctx* ctx, Batch& B, size_t njobs, size_t slot_bytes) {
  int rc;
  if ((rc = ensure(ctx->part, njobs * slot_bytes))) return rc;
  const size_t cap = ctx->cnt.cap;
  if ((rc = ensure(ctx->cnt, sizeof(int) * njobs))) return rc;
  if (ctx->cnt.cap != cap) CK(cudaMemsetAsync(ctx->cnt.p, 0, ctx->cnt.cap, ctx->stream));
  B.part = (float2*)ctx->part.p;
  B.cnt = (int*)ctx->cnt.p;
  B.part_jobs = (long long)std::min(ctx->part.cap / std::max<size_t>(1, slot_bytes), ctx->cnt.cap / sizeof(int));
  return PRONY_OK;
}

// Job list of the tensor-core products for a K split: per problem, its 128-row tiles, and per
// tile its K ranges as consecutive jobs.
// Grows the tensor-core job buffer; a reallocation invalidates the job list it held.
static int ensure_tcjobs(prony_ctx* ctx, size_t bytes) {
  const size_t cap = ctx->tcjobs.cap;
  const int rc = ensure(ctx->tcjobs, bytes);
  if (ctx->tcjobs.cap != cap) ctx->tcjob_sig.clear();
  return rc;
}

int tc_set_jobs(prony_ctx* ctx, Batch& B, int nks) {
  TcConf& T = B.tc;
  std::vector<int> sig;
  sig.reserve(3 + 2 * B.P.size());
  sig.push_back(nks);
  sig.push_back(T.gram ? T.nks_gram : 0);
  sig.push_back(T.apply ? 1 : 0);
  sig.push_back((int)B.P.size());
  for (const auto& p : B.P) {
    sig.push_back(p.n);
    sig.push_back(p.d);
  }
  int rc;
  if (ctx->tcjobs.p && sig == ctx->tcjob_sig) {
    T.njobs_ext = ctx->tcjob_next;
    T.njobs_in = ctx->tcjob_nin;
    T.njobs_gram = ctx->tcjob_ngram;
    T.njobs_apply = ctx->tcjob_napply;
    T.jobs_ext = (ToeplitzJob*)ctx->tcjobs.p;
    T.jobs_in = T.jobs_ext + T.njobs_ext;
    T.jobs_gram = T.jobs_in + T.njobs_in;
    T.jobs_apply = T.jobs_gram + T.njobs_gram;
    T.nks = nks;
  } else {
    std::vector<ToeplitzJob> jobs;
    auto add_jobs = [&](bool ext) {
      for (int i = 0; i < (int)B.P.size(); ++i) {
        const int tiles = ((ext ? B.P[i].Next : B.P[i].N) + 127) / 128;
        const int nk = std::min(nks, std::max(1, (B.P[i].N + 31) / 32));
        for (int mt = 0; mt < tiles; ++mt)
          for (int ks = 0; ks < nk; ++ks) jobs.push_back({i, mt, ks, nk});
      }
    };
    add_jobs(true);
    T.njobs_ext = (int)jobs.size();
    add_jobs(false);
    T.njobs_in = (int)jobs.size() - T.njobs_ext;
    // Grams: one row tile per problem, its K (the N rows of the tall blocks) in nks_gram ranges
    for (int i = 0; T.gram && i < (int)B.P.size(); ++i) {
      const int nk = std::min(T.nks_gram, std::max(1, (B.P[i].N + 31) / 32));
      for (int ks = 0; ks < nk; ++ks) jobs.push_back({i, 0, ks, nk});
    }
    T.njobs_gram = (int)jobs.size() - T.njobs_ext - T.njobs_in;
    // X M products: every row tile of the N rows, the whole inner dimension in one CTA
    for (int i = 0; T.apply && i < (int)B.P.size(); ++i)
      for (int mt = 0; mt < (B.P[i].N + 127) / 128; ++mt) jobs.push_back({i, mt, 0, 1});
    T.njobs_apply = (int)jobs.size() - T.njobs_ext - T.njobs_in - T.njobs_gram;
    if ((rc = ensure_tcjobs(ctx, sizeof(ToeplitzJob) * jobs.size()))) return rc;
    CK(cudaMemcpyAsync(ctx->tcjobs.p, jobs.data(), sizeof(ToeplitzJob) * jobs.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->tcjob_sig = std::move(sig);
    ctx->tcjob_next = T.njobs_ext;
    ctx->tcjob_nin = T.njobs_in;
    ctx->tcjob_ngram = T.njobs_gram;
    ctx->tcjob_napply = T.njobs_apply;
    T.jobs_ext = (ToeplitzJob*)ctx->tcjobs.p;
    T.jobs_in = T.jobs_ext + T.njobs_ext;
    T.jobs_gram = T.jobs_in + T.njobs_in;
    T.jobs_apply = T.jobs_gram + T.njobs_gram;
    T.nks = nks;
  }
  if (nks > 1 || (T.gram && T.nks_gram > 1))
    return ensure_split_ws(ctx, B, (size_t)std::max(std::max(T.njobs_ext, T.njobs_in), T.njobs_gram),
                           sizeof(float) * tc_part_floats(T.ntbox));
  return PRONY_OK;
}

int setup_tc(prony_ctx* ctx, Batch& B, int prec, int maxw) {
  TcConf& T = B.tc;
  T.on = true;
  T.kind = prec;
  const int npl = tc_planes(prec);
  T.ntbox = ((2 * maxw + 15) / 16) * 16;
  int maxnc = 0, tiles_ext = 0, tiles_in = 0;
  for (const auto& p : B.P) {
    maxnc = std::max(maxnc, (p.N + 31) / 32);
    tiles_ext += (p.Next + 127) / 128;
    tiles_in += (p.N + 127) / 128;
  }
  const size_t stage = tc_stage_bytes(prec, T.ntbox);
  const size_t avail = 227 * 1024 - 2048 - 4608;   // static shared memory of the kernel (chunk table)
  // B stages in shared memory (the kernel derives its A stages from the tensor memory that its
  // accumulator leaves free), leaving room for a window of the 2 npl split-plane tables of at
  // least 64 KB
  if (T.ntbox > 256) return PRONY_EINVAL;
  int st_max = 4;
  while (st_max > 1 && 1024 + st_max * stage + 64 * 1024 > avail) --st_max;
  // window entries per table: BF16 tables hold 2-byte entries (multiples of 8), TF32 4-byte (of 4)
  const bool bf16 = prec != PRONY_TF32X3;
  auto win_cap_for = [&](int st) {
    return (int)((avail - 1024 - st * stage) / (2 * npl * (bf16 ? 2 : 4))) & (bf16 ? ~7 : ~3);
  };
  // split K: enough CTAs to fill the GPU, every window within the shared-memory capacity, and at
  // most 512 roundings of the leading accumulator block per CTA: the FP32 accumulator in tensor
  // memory rounds once per MMA into it, one per K step (4 per chunk for BF16 planes, 8 for TF32),
  // and longer chains raise the products' rounding floor above the power iteration's default
  // tolerance.  So at most 128 K chunks per CTA for BF16 planes, 64 for TF32.
  const int max_chunks = bf16 ? 128 : 64;
  int nks_lo = std::max(1, std::min(16, (2 * 152 + tiles_in - 1) / std::max(1, tiles_in)));
  nks_lo = std::max(nks_lo, (maxnc + max_chunks - 1) / max_chunks);
  // largest window of a problem shape (it depends on n, d and the split only), computed once per
  // shape of the batch
  std::map<std::pair<int, int>, int> shapes;          // (n, d) -> a problem of that shape
  for (int i = 0; i < (int)B.P.size(); ++i) shapes.emplace(std::make_pair(B.P[i].n, B.P[i].d), i);
  std::map<std::tuple<int, int, int>, int> wmemo;      // (problem, nks, ext) -> window words
  auto window_of = [&](int i, int nks, int ext) {
    auto key = std::make_tuple(i, nks, ext);
    auto it = wmemo.find(key);
    if (it != wmemo.end()) return it->second;
    const ProbDesc& p = B.P[i];
    const int wl = max_window(p, ext ? p.n + 2 : p.n + 1, nks, bf16);
    wmemo.emplace(key, wl);
    return wl;
  };
  auto split_for = [&](int cap) {
    int nks = nks_lo;
    for (;; ++nks) {
      bool fits = true;
      for (const auto& sh : shapes) {
        const ProbDesc& p = B.P[sh.second];
        nks = std::min(nks, std::max(1, (p.N + 31) / 32));
        if (window_of(sh.second, nks, 1) > cap || window_of(sh.second, nks, 0) > cap) fits = false;
      }
      if (fits || nks >= maxnc) break;
    }
    return nks;
  };
  // Fewer B stages leave room for a longer window and so may allow a smaller split: fewer CTAs,
  // each of which pays its window load and its epilogue once.  The stage count is the largest
  // (from st_max down to two) that reaches the smallest split.
  int st_min = std::min(st_max, 2);
  if (const char* e = getenv("PRONY_TC_BSTAGES")) {   // tuning override: exactly this many B stages
    const int v = atoi(e);
    if (v >= 1) st_max = st_min = std::min(v, st_max);
  }
  int nks = INT_MAX;
  T.stages = st_max;
  for (int st = st_max; st >= st_min; --st) {
    if (win_cap_for(st) < 256) continue;
    const int k = split_for(win_cap_for(st));
    if (k < nks) {
      nks = k;
      T.stages = st;
    }
  }
  if (nks == INT_MAX) return PRONY_EINVAL;
  T.win_cap = win_cap_for(T.stages);
  T.nks_min = nks;
  T.prob_stride = tc_prob_stride(prec, T.ntbox, maxnc);
  // Grams of the tall blocks on the tensor cores, on request only (PRONY_TC_GRAM=1): the FP32
  // accumulator in tensor memory rounds once per MMA, and the Grams of CholeskyQR2, of Q = U^* T V
  // and of U^* T_l V need FP32-level accuracy: with them on the tensor cores the power iteration's
  // residual floor rises above its tolerance and C2 / C3 solves take one more iteration, which
  // costs more than the faster Grams save.  Default: the FP32 CUDA-core kernel.  Sizing when on:
  // enough CTAs to fill the GPU twice, at most 64 K chunks each; B stages as shared memory holds
  // (no window), at most 4
  {
    const char* e = getenv("PRONY_TC_GRAM");
    T.gram = e && atoi(e) == 1;
    const int np = (int)B.P.size();
    T.nks_gram = std::max(1, std::min(maxnc, (2 * 152 + np - 1) / np));
    T.nks_gram = std::max(T.nks_gram, (maxnc + 63) / 64);       // at most 64 K chunks per CTA
    const size_t gstage = tc_stage_bytes(PRONY_BF16X3, T.ntbox);
    T.gram_stages = (int)std::max<size_t>(1, std::min<size_t>(4, (avail - 1024) / gstage));
    T.gram_stride = tc_prob_stride(PRONY_BF16X3, T.ntbox, maxnc);
  }
  // X M products of the tall blocks (CholeskyQR2, the final U and V) on the tensor cores in three
  // BF16 planes, FP32-exact operands: the inner dimension is at most r0 <= 128 (four K chunks), so
  // the FP32 accumulator takes at most 16 roundings per product and plane pair.  Off with
  // PRONY_TC_APPLY=0 (the FP32 CUDA-core kernel).  B stages: up to one per K chunk of the widest X.
  // Batches whose blocks are all narrower than 32 columns keep the CUDA-core kernel: there a CTA's
  // fixed costs (tensor memory, barriers, an SM of its own) outweigh its one K chunk of MMAs (the
  // 4096 small problems of C4: 6.8 ms of tensor-core X M per step against 2.4 ms on the FP32 pipe).
  {
    const char* e = getenv("PRONY_TC_APPLY");
    T.apply = !(e && atoi(e) == 0) && maxw >= 32;
    const int maxac = (maxw + 31) / 32;
    const size_t astage = tc_stage_bytes(PRONY_BF16X3, T.ntbox);
    T.apply_stages = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::min(4, maxac), (avail - 1024) / astage));
    T.apply_stride = tc_prob_stride(PRONY_BF16X3, T.ntbox, maxac);
  }
  // batch shape signature for the tuning cache
  T.key = std::to_string(prec) + ":" + std::to_string(B.P.size()) + ":" + std::to_string(maxw) + ":" +
          std::to_string(maxnc) + ":" + std::to_string(tiles_ext) + ":" + std::to_string(tiles_in) + ":" +
          std::to_string(nks);
  auto hit = ctx->tc_tuned.find(T.key);
  T.tuned = hit != ctx->tc_tuned.end() || getenv("PRONY_TC_TUNE") != nullptr && atoi(getenv("PRONY_TC_TUNE")) == 0;
  int nks0 = hit != ctx->tc_tuned.end() ? hit->second : nks;
  if (const char* e = getenv("PRONY_TC_KSPLIT")) {    // tuning override: at least this K split
    const int v = atoi(e);
    if (v > nks0) nks0 = std::min(v, maxnc);
    T.tuned = true;
  }
  int rc;
  long long twords = 64;                              // split-plane tables (+ slack for window rounding)
  for (const auto& p : B.P) twords = std::max(twords, p.toff + 6LL * p.Gd4 + 64);
  if ((rc = ensure(ctx->tabF, 4 * (size_t)twords))) return rc;
  if ((rc = ensure(ctx->tabH, 4 * (size_t)twords))) return rc;
  B.D.tabF = (uint32_t*)ctx->tabF.p;
  B.D.tabH = (uint32_t*)ctx->tabH.p;
  // B' tiles of the products and (three BF16 planes) of the Grams share one buffer
  if ((rc = ensure(ctx->xb, (size_t)B.P.size() * (size_t)std::max(std::max(T.prob_stride, T.gram ? T.gram_stride : 0LL),
                                                                    T.apply ? T.apply_stride : 0LL))))
    return rc;
  if ((rc = ensure(ctx->tcerr, 256))) return rc;
  CK(cudaMemsetAsync(ctx->tcerr.p, 0, sizeof(int), ctx->stream));
  T.err = (int*)ctx->tcerr.p;
  return tc_set_jobs(ctx, B, nks0);
}

// One Toeplitz block product for every live problem of the batch.
int check_tc_error(prony_ctx* ctx, const Batch& B);

// The Gram X^* Z of two tall blocks (N rows) for every live problem: out (FP64, small workspace at
// out_off, leading dimension out_ld) = sum over the rows r in I_n of conj(X[r, a]) Z[r, b]; on the
// tensor cores when the batch uses them, else the FP32 CUDA-core kernel.
void gram(prony_ctx* ctx, const Batch& B, const Dev& D, int xbuf, int xshift, int xw, int zbuf, int zshift, int zw,
          long long out_off, int out_ld, cudaStream_t s) {
  const TcConf& T = B.tc;
  if (T.on && T.gram) {
    launch_xb_prep(D, zbuf, zshift, zw, ctx->xb.p, PRONY_BF16X3, T.gram_stride, s);
    cudaError_t e = launch_gram_tc(D, T.jobs_gram, T.njobs_gram, xbuf, xshift, xw, zw, out_off, out_ld, T.ntbox,
                                   T.gram_stages, ctx->xb.p, T.gram_stride, (float*)B.part, B.cnt, B.part_jobs, T.err, s);
    if (e != cudaSuccess && ctx->launch_err == cudaSuccess) ctx->launch_err = e;
  } else {
    launch_gram(D, xbuf, xshift, xw, zbuf, zshift, zw, out_off, out_ld, s);
  }
}

// OUT = X M (X in xbuf, M in the small workspace) for every live problem: on the tensor cores when
// the batch's products use them, else the FP32 CUDA-core kernel (which also serves Z - X M and the
// residual norm).
void apply(prony_ctx* ctx, const Batch& B, const Dev& D, int xbuf, int xw, int outw, long long m_off, int m_double,
           int outbuf, cudaStream_t s) {
  const TcConf& T = B.tc;
  if (T.on && T.apply && outbuf != BUF_Y) {
    cudaError_t e = launch_apply_tc(D, T.jobs_apply, T.njobs_apply, xbuf, xw, outw, m_off, m_double, outbuf, T.ntbox,
                                    T.apply_stages, ctx->xb.p, T.apply_stride, T.err, s);
    if (e != cudaSuccess && ctx->launch_err == cudaSuccess) ctx->launch_err = e;
  } else {
    launch_apply(D, xbuf, xw, outw, m_off, m_double, -1, outbuf, 0, s);
  }
}

void toeplitz_product(prony_ctx* ctx, const Batch& B, const Dev& D, int ext, int xbuf, int wsel, int ybuf, int prec,
                      cudaStream_t s, int adjoint = -1) {
  if (adjoint < 0) adjoint = ext ? 0 : 1;
  if (B.fft.on) {
    launch_toeplitz_fft(D, B.fft.maxpts, wsel == W_ONE ? 1 : B.maxw, adjoint, xbuf, wsel, ybuf, ext, s);
  } else if (B.tc.on) {
    const TcConf& T = B.tc;
    launch_xb_prep(D, xbuf, -1, wsel, ctx->xb.p, T.kind, T.prob_stride, s);
    cudaError_t e = launch_toeplitz_tc(D, ext ? T.jobs_ext : T.jobs_in, ext ? T.njobs_ext : T.njobs_in, adjoint,
                                       wsel, ybuf, ext, T.kind, T.ntbox, T.win_cap, T.stages, ctx->xb.p,
                                       T.prob_stride, (float*)B.part, B.cnt, B.part_jobs, T.err, s);
    if (e != cudaSuccess && ctx->launch_err == cudaSuccess) ctx->launch_err = e;
  } else {
    launch_toeplitz(D, ext ? B.jobs_ext : B.jobs_in, ext ? B.njobs_ext : B.njobs_in, adjoint, xbuf, wsel, ybuf, ext,
                    B.maxw, B.part, B.cnt, B.part_jobs, s);
  }
}

// Autotuner of the tensor-core products: the first product of a batch shape not seen before is
// timed (CUDA events on the context stream, one untimed and one timed launch per candidate)
// for the K splits nks_min and 2 nks_min; the faster one is kept for the batch and cached in the
// context under the shape signature.
int tc_autotune(prony_ctx* ctx, Batch& B, const Dev& D, int prec, cudaStream_t s) {
  TcConf& T = B.tc;
  std::vector<int> cand = {T.nks_min};
  if (2 * T.nks_min <= 16 && T.nks_min <= 8) cand.push_back(2 * T.nks_min);
  // room for the largest job list and split workspace first, so that no candidate reallocates them
  size_t maxjobs = 0;
  for (const auto& p : B.P) maxjobs += (size_t)2 * T.nks_min * ((p.Next + 127) / 128 + (p.N + 127) / 128);
  int rc;
  if ((rc = ensure_tcjobs(ctx, sizeof(ToeplitzJob) * maxjobs))) return rc;
  if ((rc = ensure_split_ws(ctx, B, maxjobs, sizeof(float) * tc_part_floats(T.ntbox)))) return rc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int pick = T.nks;
  for (const int c : cand) {
    if ((rc = tc_set_jobs(ctx, B, c))) break;
    toeplitz_product(ctx, B, D, 1, BUF_V, W_V, BUF_Y, prec, s);
    cudaEventRecord(e0, s);
    toeplitz_product(ctx, B, D, 1, BUF_V, W_V, BUF_Y, prec, s);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {                       // a sticky error: report it
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(e, "tensor-core autotuning");
    }
    if (ctx->launch_err != cudaSuccess) {         // this configuration does not launch: skip it
      ctx->launch_err = cudaSuccess;
      cudaGetLastError();
      continue;
    }
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = tc_set_jobs(ctx, B, pick))) return rc;
  ctx->tc_tuned[T.key] = pick;
  T.tuned = true;
  return PRONY_OK;
}

// Whether every problem of the batch is within the FFT products' limits (d <= 3, one embedded
// grid and its twiddles in a CTA's shared memory).
bool fft_fits(const Batch& B) {
  for (const auto& p : B.P)
    if (p.d > 3 || fft_points_host(p.n, p.d) + fft_length(p.n) > FFT_MAX_POINTS) return false;
  return true;
}

// FFT products: embedding length and transform offset of every problem, device tables.
int setup_fft(prony_ctx* ctx, Batch& B) {
  long long foff = 0;
  int maxpts = 0, LT = 2;
  for (auto& p : B.P) {
    p.fL = fft_length(p.n);
    const long long pts = fft_points_host(p.n, p.d);
    if (p.d > 3 || pts + p.fL > FFT_MAX_POINTS) return PRONY_EINVAL;   // line sets cover d <= 3
    p.foff = foff;
    foff += pts;
    maxpts = std::max(maxpts, (int)pts);
    LT = std::max(LT, p.fL);
  }
  int rc;
  if ((rc = ensure(ctx->fhat, sizeof(float2) * foff))) return rc;
  if ((rc = ensure(ctx->ftw, sizeof(float2) * LT))) return rc;
  CK(cudaMemcpyAsync(ctx->P.p, B.P.data(), sizeof(ProbDesc) * B.P.size(), cudaMemcpyHostToDevice, ctx->stream));
  B.D.fhat = (float2*)ctx->fhat.p;
  B.D.ftw = (float2*)ctx->ftw.p;
  B.D.fLT = LT;
  B.fft.on = true;
  B.fft.maxpts = maxpts;
  return PRONY_OK;
}

// Lay out a batch in the context workspace.  Grid samples are copied from `src`
// (host or device, per problem sample_off) into the packed grid64 buffer.
int setup_batch(prony_ctx* ctx, const std::vector<HostProb>& hp, const prony_opts& o, Batch& B) {
  const int np = (int)hp.size();
  B.P.resize(np);
  long long goff = 0, xoff = 0, yoff = 0, toff = 0;
  int maxN = 0, maxNext = 0, maxGd = 0, maxR0 = 0, maxM = 0, maxD = 0;
  long long tiles_ext = 0, tiles_in = 0;
  for (int i = 0; i < np; ++i) {
    const HostProb& h = hp[i];
    ProbDesc& p = B.P[i];
    p.d = h.d;
    p.n = h.n;
    p.m = h.m;
    p.N = (int)ipow(h.n + 1, h.d);
    p.Next = (int)ipow(h.n + 2, h.d);
    p.G = 2 * h.n + 2;
    p.Gd = (int)ipow(p.G, h.d);
    int pp = o.oversample_p < 0 ? h.m : o.oversample_p;
    p.r0 = std::min(std::min(h.m + pp, p.N), PRONY_RMAX);
    p.r0 = std::max(p.r0, h.m);
    p.grid = goff;
    p.xoff = xoff;
    p.yoff = yoff;
    p.ooff = h.out_off;
    p.Gd4 = (p.Gd + 3) & ~3;
    p.toff = toff;
    toff += 6LL * p.Gd4;
    goff += p.Gd;
    xoff += (long long)p.N * p.r0;
    yoff += (long long)p.Next * p.r0;
    maxN = std::max(maxN, p.N);
    maxNext = std::max(maxNext, p.Next);
    maxGd = std::max(maxGd, p.Gd);
    maxR0 = std::max(maxR0, p.r0);
    maxM = std::max(maxM, p.m);
    maxD = std::max(maxD, p.d);
    tiles_ext += (p.Next + 63) / 64;
    tiles_in += (p.N + 63) / 64;
  }
  SmallLay L = make_small_lay((maxR0 + 1) / 2 * 2, maxM, maxD);
  for (int i = 0; i < np; ++i) B.P[i].soff = (long long)i * L.bytes;
  // split K so that the smallest product still fills the GPU
  int nks = (int)std::max<long long>(1, std::min<long long>(304 / std::max<long long>(1, tiles_in), 16));
  nks = std::min(nks, std::max(1, maxN / 64));
  B.nks = nks;
  // job list of the FP32 CUDA-core products (the tensor-core and FFT paths build their own)
  std::vector<ToeplitzJob> jobs;
  const bool simt = o.precision == PRONY_FP32;
  for (int i = 0; simt && i < np; ++i)
    for (int mt = 0; mt < (B.P[i].Next + 63) / 64; ++mt)
      for (int ks = 0; ks < nks; ++ks) jobs.push_back({i, mt, ks, nks});
  B.njobs_ext = (int)jobs.size();
  for (int i = 0; simt && i < np; ++i)
    for (int mt = 0; mt < (B.P[i].N + 63) / 64; ++mt)
      for (int ks = 0; ks < nks; ++ks) jobs.push_back({i, mt, ks, nks});
  B.njobs_in = (int)jobs.size() - B.njobs_ext;
  B.maxw = maxR0;

  int rc;
  if ((rc = ensure(ctx->grid64, sizeof(double2) * goff))) return rc;
  if ((rc = ensure(ctx->gF, sizeof(float2) * (goff + 64)))) return rc;   // window copies may read past the end
  if ((rc = ensure(ctx->gH, sizeof(float2) * (goff + 64)))) return rc;
  if ((rc = ensure(ctx->V, sizeof(float2) * xoff))) return rc;
  if ((rc = ensure(ctx->U, sizeof(float2) * xoff))) return rc;
  if ((rc = ensure(ctx->B1, sizeof(float2) * xoff))) return rc;
  if ((rc = ensure(ctx->B2, sizeof(float2) * xoff))) return rc;
  if ((rc = ensure(ctx->Y, sizeof(float2) * yoff))) return rc;
  if ((rc = ensure(ctx->small, (size_t)L.bytes * np))) return rc;
  if ((rc = ensure(ctx->P, sizeof(ProbDesc) * np))) return rc;
  if ((rc = ensure(ctx->st, sizeof(ProbState) * np))) return rc;
  if ((rc = ensure(ctx->jobs, sizeof(ToeplitzJob) * jobs.size()))) return rc;
  if ((rc = ensure(ctx->flag, 256))) return rc;
  CK(cudaMemcpyAsync(ctx->P.p, B.P.data(), sizeof(ProbDesc) * np, cudaMemcpyHostToDevice, ctx->stream));
  if (!jobs.empty())
    CK(cudaMemcpyAsync(ctx->jobs.p, jobs.data(), sizeof(ToeplitzJob) * jobs.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
  CK(cudaMemsetAsync(ctx->small.p, 0, (size_t)L.bytes * np, ctx->stream));
  Dev& D = B.D;
  D.P = (const ProbDesc*)ctx->P.p;
  D.st = (ProbState*)ctx->st.p;
  D.nprob = np;
  D.maxN = maxN;
  D.maxNext = maxNext;
  D.maxGd = maxGd;
  D.maxR0 = maxR0;
  D.maxM = maxM;
  D.maxD = maxD;
  D.grid64 = (const double2*)ctx->grid64.p;
  D.gF = (float2*)ctx->gF.p;
  D.gH = (float2*)ctx->gH.p;
  D.V = (float2*)ctx->V.p;
  D.U = (float2*)ctx->U.p;
  D.B1 = (float2*)ctx->B1.p;
  D.B2 = (float2*)ctx->B2.p;
  D.Y = (float2*)ctx->Y.p;
  D.small = (char*)ctx->small.p;
  D.L = L;
  D.vand = o.vandermonde ? 1 : 0;
  // partials of the cross-block sums (Grams, norms, right-hand sides), one region per problem
  D.red_stride = red_bytes_per_problem(D);
  if ((rc = ensure(ctx->red, (size_t)D.red_stride * np))) return rc;
  {
    const size_t cap = ctx->rcnt.cap;
    if ((rc = ensure(ctx->rcnt, sizeof(int) * np))) return rc;
    if (ctx->rcnt.cap != cap) CK(cudaMemsetAsync(ctx->rcnt.p, 0, ctx->rcnt.cap, ctx->stream));
  }
  D.red = (char*)ctx->red.p;
  D.rcnt = (int*)ctx->rcnt.p;
  D.oob = (int*)ctx->oob.p;
  B.jobs_ext = (ToeplitzJob*)ctx->jobs.p;
  B.jobs_in = B.jobs_ext + B.njobs_ext;
  if (simt && nks > 1 &&
      (rc = ensure_split_ws(ctx, B, (size_t)std::max(B.njobs_ext, B.njobs_in), sizeof(float2) * simt_part_elems(B.maxw))))
    return rc;
  if (o.precision == PRONY_FFT32) return setup_fft(ctx, B);
  if (is_tc(o.precision) && (rc = setup_tc(ctx, B, o.precision, maxR0))) return rc;
  if (o.svd_method == 1 && fft_fits(B)) {
    // The Lanczos steps multiply by one column at a time: a tensor-core or CUDA-core product
    // costs nearly as much for one column as for twenty (the tensor-core kernel is bound by its
    // MMA issue, not by the width), an FFT product in proportion to its columns.  The Lanczos
    // vectors only start the power loop, whose products keep the chosen precision.
    if ((rc = setup_fft(ctx, B))) return rc;
    B.fft.on = false;
    B.fft.lz = true;
  }
  return PRONY_OK;
}

// CholeskyQR2 of the tall block in `xbuf` (width selector xw) into `outbuf`, through B1.
// mode: QR_PLAIN / QR_DROP / QR_RANK for the first pass; the second pass is plain.
// One pass only (plain CholeskyQR, in place) for a well-conditioned block such as the Gaussian
// start block V_0 (condition ~ (sqrt N + sqrt r0) / (sqrt N - sqrt r0), so its columns come out
// orthonormal to a few u32 after one pass).
void tall_qr1(prony_ctx* ctx, const Batch& B, int xbuf, int xw, int target, cudaStream_t s) {
  const Dev& D = B.D;
  launch_zero_small(D, D.L.gram, 16LL * D.L.LDR * D.L.LDR, s);
  gram(ctx, B, D, xbuf, -1, xw, xbuf, -1, xw, D.L.gram, D.L.LDR, s);
  launch_chol(D, xw, target, QR_PLAIN, 0.0, 0, s);
  apply(ctx, B, D, xbuf, W_IN, W_OUT, D.L.mapm, 0, xbuf, s);
}

void tall_qr(prony_ctx* ctx, const Batch& B, int xbuf, int xw, int target, int mode, double tol, int rank_mode,
             int outbuf, cudaStream_t s) {
  const Dev& D = B.D;
  launch_zero_small(D, D.L.gram, 16LL * D.L.LDR * D.L.LDR, s);
  gram(ctx, B, D, xbuf, -1, xw, xbuf, -1, xw, D.L.gram, D.L.LDR, s);
  launch_chol(D, xw, target, mode, tol, rank_mode, s);
  apply(ctx, B, D, xbuf, W_IN, W_OUT, D.L.mapm, 0, BUF_B1, s);
  launch_zero_small(D, D.L.gram, 16LL * D.L.LDR * D.L.LDR, s);
  gram(ctx, B, D, BUF_B1, -1, target, BUF_B1, -1, target, D.L.gram, D.L.LDR, s);
  launch_chol(D, target, target, QR_PLAIN, 0.0, 0, s);
  apply(ctx, B, D, BUF_B1, W_IN, W_OUT, D.L.mapm, 0, outbuf, s);
}

struct RunOut {
  int want_S = 0;
};

// Key of everything a captured loop graph bakes in: the device layout (pointers, sizes), the
// problem descriptors, the product configuration and the loop's own parameters.
std::string loop_graph_key(const Batch& B, const int* dflag, int cap, const double* params, int nparams) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  put(&B.D, sizeof(Dev));
  put(B.P.data(), sizeof(ProbDesc) * B.P.size());
  const TcConf& T = B.tc;
  const long long tc[] = {T.on, T.kind, T.ntbox, T.stages, T.win_cap, T.nks, (long long)(size_t)B.part,
                          (long long)(size_t)B.cnt, B.part_jobs, T.prob_stride, T.njobs_ext,
                          T.njobs_in, (long long)(size_t)T.jobs_ext, (long long)(size_t)T.jobs_in,
                          (long long)(size_t)T.err, B.fft.on, B.fft.lz, B.fft.maxpts, B.njobs_ext, B.njobs_in, B.nks,
                          B.maxw, (long long)(size_t)B.jobs_ext, (long long)(size_t)B.jobs_in,
                          (long long)(size_t)dflag, cap,
                          // the Gram and X M modes of the tensor-core pipeline (environment switches)
                          T.gram, T.nks_gram, T.gram_stages, T.njobs_gram, T.gram_stride,
                          (long long)(size_t)T.jobs_gram, T.apply, T.apply_stages, T.njobs_apply,
                          T.apply_stride, (long long)(size_t)T.jobs_apply};
  put(tc, sizeof(tc));
  put(params, sizeof(double) * nparams);
  return k;
}

// The whole solve as one CUDA graph, built from segments enqueued on the context stream: a
// plain segment becomes a child graph node; a loop segment becomes a WHILE conditional node
// (after a node that zeroes its body counter) whose body is the segment followed by the
// condition kernel, which reads the device flag `dflag` (nonzero once every problem has stopped)
// and caps the loop at `cap` bodies.  The handle's default value is 1: a loop runs at least once.
// Segments run in order.  Captured once per key into the context, replayed after: one graph
// launch per solve, no host round trip inside it.
struct Seg {
  bool loop;
  std::function<int()> fn;
  int cap;
  int slot;          // loop body counter slot (0: power iterations, 1: Lanczos steps)
};

int build_solve_graph(prony_ctx* ctx, const std::vector<Seg>& segs, int* dflag, const std::string& key) {
  auto& G = ctx->solve_graph;
  cudaStream_t s = ctx->stream;
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  G.key.clear();
  G.fixed_launches = 0;
  G.body_launches[0] = G.body_launches[1] = 0;
  G.has_loop[0] = G.has_loop[1] = false;
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphNode_t prev = nullptr;
  for (const Seg& seg : segs) {
    const long long before = g_launches.load();
    if (!seg.loop) {
      cudaError_t be = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
      if (be != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(be, "cudaStreamBeginCapture");
      }
      const int rc = seg.fn();
      cudaGraph_t child = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(s, &child);
      const long long n = g_launches.load() - before;
      note_launches(-n);
      G.fixed_launches += n;
      if (ce != cudaSuccess || rc) {
        if (child) cudaGraphDestroy(child);
        cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : cuda_fail(ce, "cudaStreamEndCapture");
      }
      cudaGraphNode_t node;
      const cudaError_t ae = cudaGraphAddChildGraphNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, child);
      cudaGraphDestroy(child);
      if (ae != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ae, "cudaGraphAddChildGraphNode");
      }
      prev = node;
      continue;
    }
    int* count = (int*)ctx->flag.p + 1 + seg.slot;
    cudaGraphConditionalHandle h;
    cudaMemsetParams mp = {};
    mp.dst = count;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    cudaGraphNode_t mnode, cnode;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&mnode, g, prev ? &prev : nullptr, prev ? 1 : 0, &mp);
    if (e == cudaSuccess) {
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cnode, g, &mnode, nullptr, 1, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(s, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "solve graph loop node");
    }
    const int rc = seg.fn();
    launch_loop_cond(h, dflag, count, seg.cap, s);
    cudaGraph_t body;
    const cudaError_t ce = cudaStreamEndCapture(s, &body);
    const long long n = g_launches.load() - before;
    note_launches(-n);
    G.body_launches[seg.slot] = n;
    G.has_loop[seg.slot] = true;
    if (ce != cudaSuccess) {
      // a launch inside the body failed and invalidated the capture: the parent graph (whose
      // conditional body was the capture target) is not destroyed, since the driver may not
      // handle that; it is left to the process exit
      cudaGetLastError();
      return rc ? rc : cuda_fail(ce, "cudaStreamEndCapture");
    }
    if (rc) {
      cudaGraphDestroy(g);
      return rc;
    }
    prev = cnode;
  }
  const cudaError_t ie = cudaGraphInstantiate(&G.exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    G.exec = nullptr;
    return cuda_fail(ie, "cudaGraphInstantiate");
  }
  G.key = key;
  return PRONY_OK;
}

// One replay of the solve graph; the launch statistics count its bodies as they ran.
int launch_solve_graph(prony_ctx* ctx) {
  auto& G = ctx->solve_graph;
  cudaStream_t s = ctx->stream;
  CK(cudaGraphLaunch(G.exec, s));
  CK(cudaMemcpyAsync(ctx->h_flag + 1, (int*)ctx->flag.p + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  long long n = G.fixed_launches;
  for (int k = 0; k < 2; ++k)
    if (G.has_loop[k]) n += (long long)ctx->h_flag[1 + k] * G.body_launches[k];
  note_launches(n);
  return PRONY_OK;
}

int run_batch(prony_ctx* ctx, Batch& B, const prony_opts& o, const RunOut& ro) {
  cudaStream_t s = ctx->stream;
  const Dev& D = B.D;
  const int prec = o.precision;
  const double tol_rank = o.tol_rank > 0 ? o.tol_rank : 1e-3;
  const double tol_power = o.tol_power > 0 ? o.tol_power : default_tol_power(prec);
  const int max_iter = o.max_iter > 0 ? o.max_iter : 30;
  // columns of T V whose CholeskyQR pivot falls below tol_drop^2 of the largest are dropped (the
  // noise of FP32 data); never above the rank tolerance, so that a term the rank test keeps
  // (sigma_m / sigma_1 >= tol_rank) is not lost first, and never below the FP32 resolution of the
  // Gram (3e-4 on singular-value ratios)
  const double tol_drop = std::min(1e-3, std::max(tol_rank, 3e-4));
  const double tol_lanczos = tol_rank;   // alpha, beta <= tol ||T||_F stop Algorithm 2 (Section 2.1)

  // Toeplitz launch, bracketed by events when profiling
  auto toeplitz = [&](int iter, int ext) -> int {
    int ev = -1;
    if (ctx->prof) {
      ev = (int)ctx->trecs.size() * 2;
      while ((int)ctx->events.size() < ev + 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->events.push_back(e);
      }
      ctx->trecs.push_back({ev, iter, ext, ext ? W_V : W_U});
      CK(cudaEventRecord(ctx->events[ev], s));
    }
    if (ext) toeplitz_product(ctx, B, D, 1, BUF_V, W_V, BUF_Y, prec, s);
    else toeplitz_product(ctx, B, D, 0, BUF_U, W_U, BUF_B2, prec, s);
    if (ctx->prof) CK(cudaEventRecord(ctx->events[ev + 1], s));
    return PRONY_OK;
  };
  int rc = PRONY_OK;
  if (ctx->prof) {
    ctx->trecs.clear();
    ctx->snaps.clear();
  }
  int* dflag = (int*)ctx->flag.p;
  const bool lanczos = o.svd_method == 1;
  const int lz_cap = std::max(1, D.maxR0);

  // ---- the steps of a solve, each enqueued on the context stream
  // grid copies and tables, the Philox start block (Algorithm 3: V_0)
  auto prefix = [&]() -> int {
    launch_prep(D, s);
    if (B.tc.on) launch_split_tables(D, B.tc.kind, s);
    if (B.fft.on || B.fft.lz) launch_fft_tables(D, B.fft.maxpts, s);
    launch_init_v0(D, o.seed, s);
    if (lanczos) launch_lz_start(D, s);
    return PRONY_OK;
  };
  // Algorithm 2: one Lanczos step from the first start column, full reorthogonalisation (classical
  // Gram-Schmidt twice); its right vectors start the power loop
  auto reorth = [&](int basis, int wsel) {
    for (int pass = 0; pass < 2; ++pass) {
      launch_zero_small(D, D.L.work1, 16LL * D.L.LDR * D.L.LDM, s);
      gram(ctx, B, D, basis, -1, wsel, BUF_B2, -1, W_ONE, D.L.work1, D.L.LDM, s);
      launch_apply(D, basis, wsel, W_ONE, D.L.work1, 1, BUF_B2, BUF_B2, 0, s);
    }
  };
  auto lz_product = [&](int adjoint) {                         // B2 = T B1 or T^* B1, one column
    if (B.fft.lz) launch_toeplitz_fft(D, B.fft.maxpts, 1, adjoint, BUF_B1, W_ONE, BUF_B2, 0, s);
    else toeplitz_product(ctx, B, D, 0, BUF_B1, W_ONE, BUF_B2, prec, s, adjoint);
  };
  auto lz_step = [&]() -> int {
    launch_lz_load(D, 0, s);                                       // v_k
    lz_product(0);                                                 // T v_k
    launch_lz_axpy(D, 0, s);                                       // - beta_k u_{k-1}
    reorth(BUF_U, W_LK);
    launch_lz_accept(D, 0, tol_lanczos, lz_cap, s);                // alpha_k, u_k
    launch_lz_load(D, 1, s);                                       // u_k
    lz_product(1);                                                 // T^* u_k
    launch_lz_axpy(D, 1, s);                                       // - alpha_k v_k
    reorth(BUF_V, W_LK1);
    launch_lz_accept(D, 1, tol_lanczos, lz_cap, s);                // beta_{k+1}, v_{k+1}
    CK(cudaMemsetAsync(dflag, 0xFF, sizeof(int), s));
    launch_lz_all_done(D, dflag, s);
    return PRONY_OK;
  };
  // V_0 orthonormal (or the Lanczos right vectors), then Y = T V_0
  auto start = [&]() -> int {
    if (lanczos) launch_lz_finish(D, s);
    else tall_qr1(ctx, B, BUF_V, W_R0, W_V, s);
    return toeplitz(0, 1);
  };
  // one power iteration (Algorithm 3); dflag ends nonzero when every problem has stopped
  auto iteration = [&](int it) -> int {
    // U = qr(T V_{k-1})  (rows I_n of Y)
    tall_qr(ctx, B, BUF_Y, W_V, W_U, QR_DROP, tol_drop, 0, BUF_U, s);
    // Vbar = T^* U
    if ((rc = toeplitz(it, 0))) return rc;
    // V = qr(Vbar), column pivoting and the rank test on a problem's first iteration
    tall_qr(ctx, B, BUF_B2, W_U, W_V, QR_AUTO, tol_rank, o.rank_mode, BUF_V, s);
    // Y = T V over the box {0..n+1}^d
    if ((rc = toeplitz(it, 1))) return rc;
    // Q = U^* (T V), ||T V - U Q||_F
    launch_zero_small(D, D.L.q, 16LL * D.L.LDR * D.L.LDM, s);
    gram(ctx, B, D, BUF_U, -1, W_U, BUF_Y, -1, W_V, D.L.q, D.L.LDM, s);
    launch_apply(D, BUF_U, W_U, W_V, D.L.q, 1, BUF_Y, -1, 1, s);
    CK(cudaMemsetAsync(dflag, 0xFF, sizeof(int), s));
    launch_check(D, tol_power, max_iter, dflag, s);
    return PRONY_OK;
  };
  // finishing steps, for every problem that has not failed
  auto finish = [&]() -> int {
    launch_reset_done(D, s);
    // M_l = U^* Y_l  with Y_l the rows k + e_l of the last product Y = T V
    launch_zero_small(D, D.L.mproj, 16LL * D.maxD * D.L.LDR * D.L.LDM, s);
    for (int l = 0; l < D.maxD; ++l)
      gram(ctx, B, D, BUF_U, -1, W_U, BUF_Y, l, W_V, D.L.mproj + 16LL * l * D.L.LDR * D.L.LDM, D.L.LDM, s);
    launch_svd_S(D, s);
    if (ro.want_S) {
      // phase-canonical basis: argmax over V V_Q, then rotate U_Q, V_Q, S_l
      apply(ctx, B, D, BUF_V, W_V, W_V, D.L.vq, 1, BUF_B1, s);
      launch_zero_small(D, D.L.argmx, 8LL * D.L.LDM, s);
      launch_argmax(D, BUF_B1, s);
      launch_canon(D, s);
      apply(ctx, B, D, BUF_V, W_V, W_V, D.L.vq, 1, BUF_B1, s);   // V_final
      apply(ctx, B, D, BUF_U, W_U, W_V, D.L.uq, 1, BUF_B2, s);   // U_final
    }
    launch_eig_t(D, o.seed, s);
    launch_zero_small(D, D.L.rhs, 16LL * D.L.LDM, s);
    launch_rhs(D, 0, s);
    launch_solve_c(D, s);
    launch_rhs(D, 1, s);
    return PRONY_OK;
  };

  // ---- as one graph (the usual case), or step by step from the host: with profiling (events
  // around every product) and on the first call for a batch shape (the product autotuner times
  // candidates between the start block and the first product)
  const bool graph = !ctx->prof && !(B.tc.on && !B.tc.tuned);
  if (graph) {
    const double par[] = {tol_rank, tol_power, tol_drop, (double)max_iter, (double)prec, (double)o.svd_method,
                          (double)o.rank_mode, (double)o.vandermonde, (double)ro.want_S};
    std::string key = loop_graph_key(B, dflag, max_iter, par, (int)(sizeof(par) / sizeof(par[0])));
    key.append((const char*)&o.seed, sizeof(o.seed));
    if (!ctx->solve_graph.exec || key != ctx->solve_graph.key) {
      std::vector<Seg> segs;
      segs.push_back({false, prefix, 0, 0});
      if (lanczos) segs.push_back({true, lz_step, lz_cap, 1});
      segs.push_back({false, start, 0, 0});
      segs.push_back({true, [&]() { return iteration(1); }, max_iter, 0});
      segs.push_back({false, finish, 0, 0});
      if ((rc = build_solve_graph(ctx, segs, dflag, key))) return rc;
    }
    if ((rc = launch_solve_graph(ctx))) return rc;
    CK(cudaGetLastError());
    return check_tc_error(ctx, B);
  }
  prefix();
  if (lanczos) {
    for (int step = 0; step < lz_cap; ++step) {
      if ((rc = lz_step())) return rc;
      CK(cudaMemcpyAsync(ctx->h_flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*ctx->h_flag != 0) break;
    }
  }
  if (B.tc.on && !B.tc.tuned && (rc = tc_autotune(ctx, B, D, prec, s))) return rc;
  if ((rc = start())) return rc;
  if (ctx->prof) {
    ctx->snaps.emplace_back(D.nprob);
    CK(cudaMemcpyAsync(ctx->snaps.back().data(), D.st, sizeof(ProbState) * D.nprob, cudaMemcpyDeviceToHost, s));
  }
  for (int it = 1; it <= max_iter; ++it) {
    if ((rc = iteration(it))) return rc;
    CK(cudaMemcpyAsync(ctx->h_flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (ctx->prof) {
      ctx->snaps.emplace_back(D.nprob);
      CK(cudaMemcpyAsync(ctx->snaps.back().data(), D.st, sizeof(ProbState) * D.nprob, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (*ctx->h_flag != 0) break;
  }
  if (ctx->prof) {
    // accumulate durations and algorithmic work of the Toeplitz launches of this solve
    CK(cudaStreamSynchronize(s));
    for (const auto& r : ctx->trecs) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ctx->events[r.ev], ctx->events[r.ev + 1]));
      const auto& before = ctx->snaps[r.iter > 0 ? r.iter - 1 : 0];
      const auto& after = ctx->snaps[r.iter];
      double fl = 0.0, by = 0.0;
      for (int p = 0; p < D.nprob; ++p) {
        if (r.iter > 0 && before[p].done) continue;
        const ProbDesc& q = B.P[p];
        int w = r.iter == 0 ? q.r0 : (r.ext ? after[p].wv : after[p].wu);
        double rows = r.ext ? q.Next : q.N;
        if (B.fft.on) {
          // transforms as computed: per axis the pruned lines, 5 L log2 L flops each, forward and
          // inverse, plus the pointwise product (6 flops per point)
          const int L = q.fL, K = r.ext ? q.n + 2 : q.n + 1;
          double lines = 0.0, lg = std::log2((double)L);
          for (int ax = 0; ax < q.d; ++ax)
            lines += std::pow((double)(q.n + 1), ax) * std::pow((double)L, q.d - 1 - ax) +
                     std::pow((double)K, ax) * std::pow((double)L, q.d - 1 - ax);
          fl += w * (5.0 * L * lg * lines + 6.0 * std::pow((double)L, q.d));
          by += 8.0 * q.N * w + 8.0 * rows * w + 8.0 * (double)fft_points_host(q.n, q.d);
        } else {
          fl += 8.0 * rows * q.N * w;
          by += 8.0 * q.Gd + 8.0 * q.N * w + 8.0 * rows * w;
        }
      }
      ctx->stats.tc_ksplit = B.tc.on ? B.tc.nks : 0;
      ctx->stats.tc_bstages = B.tc.on ? B.tc.stages : 0;
      ctx->stats.toeplitz_launches += 1;
      ctx->stats.toeplitz_ms += ms;
      ctx->stats.toeplitz_flops += fl;
      ctx->stats.toeplitz_bytes += by;
    }
  }
  finish();
  CK(cudaGetLastError());
  return check_tc_error(ctx, B);
}

int read_states(prony_ctx* ctx, const Batch& B, prony_info* infos, int* worst) {
  const int np = B.D.nprob;
  ctx->h_st.resize(np);
  CK(cudaMemcpyAsync(ctx->h_st.data(), B.D.st, sizeof(ProbState) * np, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int w = PRONY_OK;
  for (int i = 0; i < np; ++i) {
    const ProbState& s = ctx->h_st[i];
    if (infos) {
      prony_info& I = infos[i];
      I.status = s.status;
      I.rank_detected = s.rank_det;
      I.rank_used = s.rank_used;
      I.power_iters = s.iter;
      I.normT = std::sqrt(std::max(0.0, s.normT2));
      I.power_resid = s.normT2 > 0 ? std::sqrt(std::max(0.0, s.resid2) / s.normT2) : 0.0;
      I.ls_resid = s.normf2 > 0 ? std::sqrt(std::max(0.0, s.ls_num2) / s.normf2) : 0.0;
      I.sigma_ratio = s.sigma_ratio;
      I.lanczos_steps = s.lk;
    }
    if (s.status != PRONY_OK && (w == PRONY_OK || s.status < w)) w = s.status;
  }
  *worst = w;
  return PRONY_OK;
}

prony_opts resolve_opts(const prony_opts* o) {
  prony_opts r;
  prony_default_opts(&r);
  if (o) r = *o;
  return r;
}

int check_precision(int prec) {
  return (prec == PRONY_FP32 || prec == PRONY_FFT32 || is_tc(prec)) ? PRONY_OK : PRONY_EINVAL;
}

// Error flags of the kernels: a failed workspace bound check (any kernel; the access was skipped,
// the split-K and cross-block counters are cleared for the next call) and the tensor-core kernels'
// bounded waits or window overflow.
int check_tc_error(prony_ctx* ctx, const Batch& B) {
  int oob = 0;
  CK(cudaMemcpyAsync(&oob, ctx->oob.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (oob) {
    CK(cudaMemsetAsync(ctx->oob.p, 0, sizeof(int), ctx->stream));
    if (ctx->cnt.p) CK(cudaMemsetAsync(ctx->cnt.p, 0, ctx->cnt.cap, ctx->stream));
    if (ctx->rcnt.p) CK(cudaMemsetAsync(ctx->rcnt.p, 0, ctx->rcnt.cap, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    g_err = "internal workspace bound check failed at site " + std::to_string(oob);
    return PRONY_ECUDA;
  }
  if (!B.tc.on) return PRONY_OK;
  if (ctx->launch_err != cudaSuccess) {
    const cudaError_t e = ctx->launch_err;
    ctx->launch_err = cudaSuccess;
    g_err = std::string("tensor-core Toeplitz launch: ") + cudaGetErrorString(e);
    return PRONY_ECUDA;
  }
  int h = 0;
  CK(cudaMemcpyAsync(&h, B.tc.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) {
    g_err = "tensor-core Toeplitz kernel reported error " + std::to_string(h);
    return PRONY_ECUDA;
  }
  return PRONY_OK;
}

// Copy problem grids to the packed device buffer (host or device source).
// Samples into the packed grid buffer: one copy per run of problems whose grids are adjacent
// both in the caller's array and in the buffer (the usual packed layout is a single copy).
int load_grids(prony_ctx* ctx, const Batch& B, const std::vector<HostProb>& hp, const prony_c128* src, bool device) {
  size_t i = 0;
  while (i < hp.size()) {
    const long long s0 = hp[i].sample_off, d0 = B.P[i].grid;
    long long len = B.P[i].Gd;
    size_t j = i + 1;
    while (j < hp.size() && hp[j].sample_off == s0 + len && B.P[j].grid == d0 + len) len += B.P[j++].Gd;
    CK(cudaMemcpyAsync((double2*)ctx->grid64.p + d0, src + s0, sizeof(double2) * len,
                       device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    i = j;
  }
  return PRONY_OK;
}

}  // namespace

// ============================================================================= C ABI
extern "C" {

void prony_default_opts(prony_opts* o) {
  if (!o) return;
  o->precision = PRONY_BF16X3;
  o->oversample_p = -1;
  o->tol_rank = 0.0;
  o->tol_power = 0.0;
  o->max_iter = 0;
  o->seed = 2012114300ull;
  o->rank_mode = 0;
  o->vandermonde = 0;
  o->svd_method = 0;
}

const char* prony_status_string(int s) {
  switch (s) {
    case PRONY_OK: return "ok";
    case PRONY_EINVAL: return "invalid argument";
    case PRONY_ERANK: return "numerical rank below m";
    case PRONY_ENOCONV: return "iteration cap reached";
    case PRONY_ENAN: return "non-finite data";
    case PRONY_ECUDA: return "CUDA error";
    case PRONY_ENOMEM: return "device allocation failed";
    default: return "unknown status";
  }
}

const char* prony_last_error(void) { return g_err.c_str(); }

int prony_ctx_create(prony_ctx** out, int device) {
  if (!out) return PRONY_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return PRONY_EINVAL;
  CK(cudaSetDevice(device));
  prony_ctx* c = new prony_ctx();
  c->device = device;
  e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate"); }
  e = cudaMallocHost(&c->h_flag, 256);
  if (e != cudaSuccess) { cudaStreamDestroy(c->stream); delete c; return cuda_fail(e, "cudaMallocHost"); }
  if (ensure(c->oob, 256) != PRONY_OK || cudaMemsetAsync(c->oob.p, 0, 256, c->stream) != cudaSuccess) {
    if (c->oob.p) cudaFree(c->oob.p);
    cudaFreeHost(c->h_flag);
    cudaStreamDestroy(c->stream);
    delete c;
    return PRONY_ENOMEM;
  }
  *out = c;
  return PRONY_OK;
}

int prony_ctx_destroy(prony_ctx* c) {
  if (!c) return PRONY_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  DBuf* bufs[] = {&c->grid64, &c->gF, &c->gH, &c->V, &c->U, &c->B1, &c->B2, &c->Y, &c->small, &c->P,
                  &c->st, &c->jobs, &c->flag, &c->tout, &c->cout, &c->misc, &c->misc2, &c->misc3,
                  &c->xb, &c->tabF, &c->tabH, &c->tcjobs, &c->tcerr, &c->lmws, &c->part, &c->cnt, &c->red,
                  &c->rcnt, &c->oob};
  if (c->lm_exec) cudaGraphExecDestroy(c->lm_exec);
  if (c->solve_graph.exec) cudaGraphExecDestroy(c->solve_graph.exec);
  for (DBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  cudaStreamDestroy(c->stream);
  delete c;
  return PRONY_OK;
}

int prony_set_profiling(prony_ctx* c, int enable) {
  if (!c) return PRONY_EINVAL;
  c->prof = enable != 0;
  c->stats = prony_stats{};
  c->launch_base = g_launches.load();
  return PRONY_OK;
}

int prony_get_stats(prony_ctx* c, prony_stats* out) {
  if (!c || !out) return PRONY_EINVAL;
  *out = c->stats;
  out->launches = g_launches.load() - c->launch_base;
  return PRONY_OK;
}

static int solve_batched_impl(prony_ctx* ctx, int P, const int* d, const int* n, const int* m,
                              const long long* sample_off, const prony_c128* samples, bool dev_samples,
                              const long long* out_off, double* t_out, prony_c128* c_out, bool dev_out,
                              prony_info* infos, const prony_opts* opts, cudaStream_t user_stream) {
  if (!ctx || P <= 0 || !d || !n || !m || !sample_off || !samples || !out_off || !t_out || !c_out)
    return PRONY_EINVAL;
  prony_opts o = resolve_opts(opts);
  if (check_precision(o.precision)) return PRONY_EINVAL;
  CK(cudaSetDevice(ctx->device));
  std::vector<HostProb> hp(P);
  long long total_terms = 0;
  for (int i = 0; i < P; ++i) {
    hp[i] = {d[i], n[i], m[i], sample_off[i], out_off[i]};
    if (validate(hp[i])) return PRONY_EINVAL;
    total_terms = std::max(total_terms, out_off[i] + m[i]);
  }
  if (user_stream) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, user_stream));
    CK(cudaStreamWaitEvent(ctx->stream, ev, 0));
    cudaEventDestroy(ev);
  }
  Batch B;
  int rc = setup_batch(ctx, hp, o, B);
  if (rc) return rc;
  if ((rc = load_grids(ctx, B, hp, samples, dev_samples))) return rc;
  RunOut ro;
  if ((rc = run_batch(ctx, B, o, ro))) return rc;
  int maxd = B.D.maxD;
  double* tdev = t_out;
  double2* cdev = (double2*)c_out;
  if (!dev_out) {
    if ((rc = ensure(ctx->tout, sizeof(double) * total_terms * maxd))) return rc;
    if ((rc = ensure(ctx->cout, sizeof(double2) * total_terms))) return rc;
    tdev = (double*)ctx->tout.p;
    cdev = (double2*)ctx->cout.p;
  }
  launch_gather_out(B.D, tdev, cdev, ctx->stream);
  CK(cudaGetLastError());
  int worst = PRONY_OK;
  if ((rc = read_states(ctx, B, infos, &worst))) return rc;
  if (!dev_out) {
    // rows of maxd entries; a problem writes its first d of each row only
    std::vector<double> th(total_terms * maxd);
    std::vector<double2> ch(total_terms);
    CK(cudaMemcpy(th.data(), tdev, sizeof(double) * total_terms * maxd, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ch.data(), cdev, sizeof(double2) * total_terms, cudaMemcpyDeviceToHost));
    for (int i = 0; i < P; ++i) {
      for (int j = 0; j < m[i]; ++j)
        std::memcpy(t_out + (out_off[i] + j) * maxd, th.data() + (out_off[i] + j) * maxd, sizeof(double) * d[i]);
      std::memcpy(c_out + out_off[i], ch.data() + out_off[i], sizeof(double2) * m[i]);
    }
  } else if (user_stream) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, ctx->stream));
    CK(cudaStreamWaitEvent(user_stream, ev, 0));
    cudaEventDestroy(ev);
    CK(cudaStreamSynchronize(user_stream));
  }
  return worst;
}

int prony_solve_batched(prony_ctx* ctx, int P, const int* d, const int* n, const int* m,
                        const long long* sample_off, const prony_c128* samples, const long long* out_off,
                        double* t_out, prony_c128* c_out, prony_info* infos, const prony_opts* opts) {
  return solve_batched_impl(ctx, P, d, n, m, sample_off, samples, false, out_off, t_out, c_out, false, infos, opts,
                            nullptr);
}

int prony_solve_batched_dev(prony_ctx* ctx, int P, const int* d, const int* n, const int* m,
                            const long long* sample_off, const prony_c128* samples_dev, const long long* out_off,
                            double* t_out_dev, prony_c128* c_out_dev, prony_info* infos, const prony_opts* opts,
                            void* stream) {
  return solve_batched_impl(ctx, P, d, n, m, sample_off, samples_dev, true, out_off, t_out_dev, c_out_dev, true,
                            infos, opts, (cudaStream_t)stream);
}

int prony_solve(prony_ctx* ctx, const prony_c128* samples, int d, int n, int m, const prony_opts* opts,
                double* t_out, prony_c128* c_out, prony_info* info) {
  long long zero = 0;
  return solve_batched_impl(ctx, 1, &d, &n, &m, &zero, samples, false, &zero, t_out, c_out, false, info, opts,
                            nullptr);
}

int prony_build_S(prony_ctx* ctx, const prony_c128* samples, int d, int n, int m, const prony_opts* opts,
                  prony_c128* S_out, double* sigma_out, prony_c128* U_out, prony_c128* V_out, prony_info* info) {
  if (!ctx || !samples || !S_out || !sigma_out) return PRONY_EINVAL;
  prony_opts o = resolve_opts(opts);
  if (check_precision(o.precision)) return PRONY_EINVAL;
  CK(cudaSetDevice(ctx->device));
  std::vector<HostProb> hp = {{d, n, m, 0, 0}};
  if (validate(hp[0])) return PRONY_EINVAL;
  Batch B;
  int rc = setup_batch(ctx, hp, o, B);
  if (rc) return rc;
  if ((rc = load_grids(ctx, B, hp, samples, false))) return rc;
  RunOut ro;
  ro.want_S = 1;
  if ((rc = run_batch(ctx, B, o, ro))) return rc;
  const SmallLay& L = B.D.L;
  std::vector<char> small(L.bytes);
  CK(cudaMemcpyAsync(small.data(), ctx->small.p, L.bytes, cudaMemcpyDeviceToHost, ctx->stream));
  const long long N = B.P[0].N;
  std::vector<double2> Uh, Vh;
  if (U_out || V_out) {
    if ((rc = ensure(ctx->misc, sizeof(double2) * N * m))) return rc;
    if (U_out) {
      launch_copy_cols(B.D, BUF_B2, W_V, (double2*)ctx->misc.p, ctx->stream);
      CK(cudaMemcpyAsync(U_out, ctx->misc.p, sizeof(double2) * N * m, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    if (V_out) {
      launch_copy_cols(B.D, BUF_B1, W_V, (double2*)ctx->misc.p, ctx->stream);
      CK(cudaMemcpyAsync(V_out, ctx->misc.p, sizeof(double2) * N * m, cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  int worst = PRONY_OK;
  if ((rc = read_states(ctx, B, info, &worst))) return rc;
  const int w = ctx->h_st[0].wv;
  const double2* S = (const double2*)(small.data() + L.S);
  const double* sg = (const double*)(small.data() + L.sigma);
  for (int l = 0; l < d; ++l)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double2 v = (i < w && j < w) ? S[(size_t)l * L.LDM * L.LDM + i * L.LDM + j] : make_double2(0.0, 0.0);
        S_out[((size_t)l * m + i) * m + j] = {v.x, v.y};
      }
  for (int i = 0; i < m; ++i) sigma_out[i] = i < w ? sg[i] : 0.0;
  return worst;
}

int prony_small_steps(prony_ctx* ctx, int d, int m, int a, const prony_c128* Q, const prony_c128* M,
                      unsigned long long seed, int jacobi_cap, int eigqr_cap, double* sigma_out, prony_c128* S_out,
                      prony_c128* z_out, double* t_out, int* status_out) {
  if (!ctx || !Q || !M || !sigma_out || !S_out || !z_out || !t_out || d < 1 || d > PRONY_DMAX || m < 1 ||
      m > PRONY_MMAX || a < m || a > PRONY_RMAX)
    return PRONY_EINVAL;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  // one problem whose power loop has "ended" with U of width a and V of width m: the state and
  // the small workspace are written directly, no tall block or product is involved
  ProbDesc pd{};
  pd.d = d;
  pd.m = m;
  pd.r0 = a;
  pd.n = 1;
  pd.N = a;
  ProbState st{};
  st.wu = a;
  st.wv = m;
  st.rank_used = m;
  st.rank_det = m;
  const SmallLay L = make_small_lay((a + 1) / 2 * 2, m, d);
  int rc;
  if ((rc = ensure(ctx->small, (size_t)L.bytes))) return rc;
  if ((rc = ensure(ctx->P, sizeof(ProbDesc)))) return rc;
  if ((rc = ensure(ctx->st, sizeof(ProbState)))) return rc;
  CK(cudaMemsetAsync(ctx->small.p, 0, (size_t)L.bytes, s));
  CK(cudaMemcpyAsync(ctx->P.p, &pd, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->st.p, &st, sizeof(ProbState), cudaMemcpyHostToDevice, s));
  char* sb = (char*)ctx->small.p;
  // Q (a x m) and U^* T_l V (a x m each), row-major with leading dimension LDM
  CK(cudaMemcpy2DAsync(sb + L.q, sizeof(double2) * L.LDM, Q, sizeof(prony_c128) * m, sizeof(prony_c128) * m, a,
                       cudaMemcpyHostToDevice, s));
  for (int l = 0; l < d; ++l)
    CK(cudaMemcpy2DAsync(sb + L.mproj + 16LL * l * L.LDR * L.LDM, sizeof(double2) * L.LDM, M + (size_t)l * a * m,
                         sizeof(prony_c128) * m, sizeof(prony_c128) * m, a, cudaMemcpyHostToDevice, s));
  Dev D{};
  D.P = (const ProbDesc*)ctx->P.p;
  D.st = (ProbState*)ctx->st.p;
  D.nprob = 1;
  D.maxN = a;
  D.maxR0 = a;
  D.maxM = m;
  D.maxD = d;
  D.small = sb;
  D.L = L;
  D.cap_jacobi = jacobi_cap;
  D.cap_eigqr = eigqr_cap;
  launch_svd_S(D, s);
  launch_eig_t(D, seed, s);
  CK(cudaGetLastError());
  std::vector<char> h(L.bytes);
  CK(cudaMemcpyAsync(h.data(), sb, L.bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, ctx->st.p, sizeof(ProbState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double* sg = (const double*)(h.data() + L.sigma);
  const double2* S = (const double2*)(h.data() + L.S);
  const double2* z = (const double2*)(h.data() + L.zraw);
  const double* t = (const double*)(h.data() + L.t);
  for (int i = 0; i < m; ++i) sigma_out[i] = sg[i];
  for (int l = 0; l < d; ++l)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double2 v = S[(size_t)l * L.LDM * L.LDM + (size_t)i * L.LDM + j];
        S_out[((size_t)l * m + i) * m + j] = {v.x, v.y};
      }
  for (int j = 0; j < m; ++j)
    for (int l = 0; l < d; ++l) {
      const double2 v = z[j * PRONY_DMAX + l];
      z_out[(size_t)j * d + l] = {v.x, v.y};
      t_out[(size_t)j * d + l] = t[j * PRONY_DMAX + l];
    }
  if (status_out) *status_out = st.status;
  return PRONY_OK;
}

int prony_eval(prony_ctx* ctx, const double* t, const prony_c128* c, int m, int d, const int* k, int K,
               prony_c128* f_out) {
  if (!ctx || !t || !c || !k || !f_out || m < 1 || m > PRONY_MMAX || d < 1 || d > PRONY_DMAX || K < 0)
    return PRONY_EINVAL;
  if (K == 0) return PRONY_OK;
  CK(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = ensure(ctx->misc, sizeof(double) * m * d + sizeof(double2) * m))) return rc;
  if ((rc = ensure(ctx->misc2, sizeof(int) * (size_t)K * d))) return rc;
  if ((rc = ensure(ctx->misc3, sizeof(double2) * (size_t)K))) return rc;
  double* td = (double*)ctx->misc.p;
  double2* cd = (double2*)((char*)ctx->misc.p + ((sizeof(double) * m * d + 15) / 16 * 16));
  CK(cudaMemcpyAsync(td, t, sizeof(double) * m * d, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(cd, c, sizeof(double2) * m, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->misc2.p, k, sizeof(int) * (size_t)K * d, cudaMemcpyHostToDevice, ctx->stream));
  launch_eval_points(td, cd, m, d, (const int*)ctx->misc2.p, K, (double2*)ctx->misc3.p, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(f_out, ctx->misc3.p, sizeof(double2) * (size_t)K, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PRONY_OK;
}

static long long box_count(int d, const int* len) {
  long long K = 1;
  for (int l = 0; l < d; ++l) {
    if (len[l] < 0) return -1;
    K *= len[l];
  }
  return K;
}

int prony_expsum_fwd_dev(prony_ctx* ctx, const double* t_dev, const void* c_dev, int m, int d, const int* lo,
                         const int* len, void* f_dev, void* stream) {
  if (!ctx || !t_dev || !c_dev || !f_dev || !lo || !len || m < 1 || m > PRONY_MMAX || d < 1 || d > PRONY_DMAX)
    return PRONY_EINVAL;
  long long K = box_count(d, len);
  if (K < 0) return PRONY_EINVAL;
  if (K == 0) return PRONY_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  launch_expsum_fwd(t_dev, (const float2*)c_dev, m, d, lo, len, K, (float2*)f_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return PRONY_OK;
}

int prony_refine_lm_dev(prony_ctx* ctx, double* t_dev, prony_c128* c_dev, int m, int d, const int* lo,
                        const int* len, const void* y_dev, int iters, double lambda0, double* loss_dev, void* stream) {
  if (!ctx || !t_dev || !c_dev || !y_dev || !lo || !len || m < 1 || m > PRONY_MMAX || d < 1 || d > PRONY_DMAX ||
      iters < 0 || m * (d + 2) > PRONY_LM_PMAX || !(lambda0 > 0.0))
    return PRONY_EINVAL;
  const long long K = box_count(d, len);
  if (K <= 0) return PRONY_EINVAL;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  if (iters == 0) return PRONY_OK;
  int rc;
  if ((rc = ensure(ctx->lmws, (size_t)lm_workspace_bytes(m, d)))) return rc;
  prony_ctx::LmKey k{};
  k.t = t_dev; k.c = c_dev; k.y = y_dev; k.loss = loss_dev; k.ws = ctx->lmws.p;
  k.m = m; k.d = d; k.iters = iters; k.lambda0 = lambda0;
  for (int l = 0; l < d; ++l) { k.lo[l] = lo[l]; k.len[l] = len[l]; }
  if (!ctx->lm_exec || std::memcmp(&k, &ctx->lm_key, sizeof(k)) != 0) {
    if (ctx->lm_exec) {
      cudaGraphExecDestroy(ctx->lm_exec);
      ctx->lm_exec = nullptr;
    }
    CK(lm_set_attributes(m, d));
    // capture on the context stream (never the legacy default stream), launch on `s`
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    launch_refine_lm(t_dev, (double2*)c_dev, m, d, lo, len, K, (const float2*)y_dev, iters, lambda0, loss_dev,
                     ctx->lmws.p, ctx->stream);
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture(ctx->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&ctx->lm_exec, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    ctx->lm_key = k;
  } else {
    note_launches(1 + (long long)LM_LAUNCHES_PER_STEP * iters);
  }
  CK(cudaGraphLaunch(ctx->lm_exec, s));
  CK(cudaStreamSynchronize(s));
  return PRONY_OK;
}

int prony_expsum_bwd_dev(prony_ctx* ctx, const double* t_dev, const void* c_dev, int m, int d, const int* lo,
                         const int* len, const void* g_dev, double* grad_t_dev, void* grad_c_dev, void* stream) {
  if (!ctx || !t_dev || !c_dev || !g_dev || !grad_t_dev || !grad_c_dev || !lo || !len || m < 1 ||
      m > PRONY_MMAX || d < 1 || d > PRONY_DMAX)
    return PRONY_EINVAL;
  long long K = box_count(d, len);
  if (K < 0) return PRONY_EINVAL;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  int rc;
  if ((rc = ensure(ctx->misc3, sizeof(double) * m * (2 + d)))) return rc;
  CK(cudaMemsetAsync(ctx->misc3.p, 0, sizeof(double) * m * (2 + d), s));
  if (K > 0) launch_expsum_bwd(t_dev, (const float2*)c_dev, m, d, lo, len, K, (const float2*)g_dev,
                               (double*)ctx->misc3.p, s);
  launch_expsum_bwd_finish((const double*)ctx->misc3.p, m, d, grad_t_dev, (float2*)grad_c_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return PRONY_OK;
}

int prony_toeplitz_mm_dev(prony_ctx* ctx, const prony_c128* grid_dev, int d, int n, const void* X_dev, int r, int L,
                          int adjoint, int precision, void* Y_dev, void* stream) {
  if (!ctx || !grid_dev || !X_dev || !Y_dev || d < 1 || d > PRONY_DMAX || n < 1 || r < 1 || r > PRONY_RMAX)
    return PRONY_EINVAL;
  if (L != n + 1 && L != n + 2) return PRONY_EINVAL;
  if (adjoint && L != n + 1) return PRONY_EINVAL;
  if (check_precision(precision)) return PRONY_EINVAL;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  std::vector<HostProb> hp = {{d, n, 1, 0, 0}};
  if (std::pow((double)(n + 1), d) > 2.0e8 || r > (long long)ipow(n + 1, d)) return PRONY_EINVAL;
  prony_opts o;
  prony_default_opts(&o);
  o.oversample_p = r - 1;
  o.precision = precision;
  Batch B;
  // ensure the stream order: ctx work after the caller's stream
  if (stream) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, s));
    CK(cudaStreamWaitEvent(ctx->stream, ev, 0));
    cudaEventDestroy(ev);
  }
  int rc = setup_batch(ctx, hp, o, B);
  if (rc) return rc;
  B.P[0].r0 = r;
  CK(cudaMemcpyAsync(ctx->P.p, B.P.data(), sizeof(ProbDesc), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->grid64.p, grid_dev, sizeof(double2) * B.P[0].Gd, cudaMemcpyDeviceToDevice, ctx->stream));
  launch_prep(B.D, ctx->stream);
  if (B.tc.on) launch_split_tables(B.D, B.tc.kind, ctx->stream);
  if (B.fft.on) launch_fft_tables(B.D, B.fft.maxpts, ctx->stream);
  // operate directly on the caller's buffers: X as V (ld N), Y as Y (ld L^d)
  Dev D = B.D;
  D.V = (float2*)X_dev;
  D.Y = (float2*)Y_dev;
  D.B2 = (float2*)Y_dev;
  const int y_ext = (L == n + 2);
  toeplitz_product(ctx, B, D, y_ext, BUF_V, W_R0, y_ext ? BUF_Y : BUF_B2, precision, ctx->stream, adjoint);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return check_tc_error(ctx, B);
}

}  // extern "C"
