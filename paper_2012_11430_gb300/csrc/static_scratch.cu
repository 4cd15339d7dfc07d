// prony_toeplitz_mm_static: the Toeplitz block product with no device allocation.
//
// Some callers cannot let a library call cudaMalloc: host code whose device memory is
// fixed up front by its own allocator or memory budget, and latency-critical loops
// where cudaMalloc / cudaFree may synchronise the device and stall other streams.
// This entry point keeps all of its scratch -- the problem descriptor and iteration
// state, the job list, and the complex64 copies of the sample grid that the product
// kernel reads -- in one file-scope device array of fixed size, so it needs no context
// and allocates nothing.  Inputs and outputs are the caller's device buffers.
//
// The array is a static device symbol: every GPU that loads the library holds it
// (PRONY_STATIC_SCRATCH_BYTES) until the process exits.  In host code its name stands
// for a host-side shadow, not a device address, so every call looks up its device address
// on the current device with cudaGetSymbolAddress (a cheap lookup once the module is loaded;
// nothing is cached, so a reset device or another context never sees a stale address).  The
// first call on a device loads the library's module there and reserves the array, which may
// synchronise: make it once as a warm-up, outside latency-critical loops and before any stream
// capture.  All calls share the one array: calls that overlap on the GPU (for example on two
// streams) race on it.
//
// The product runs without a K split (one CTA per row tile), so it needs no partial-sum
// workspace and its sums have one fixed order.
#include "common.cuh"
#include "../../include/prony.h"

#include <algorithm>

namespace {

constexpr long long kMaxJobs = 65536 - 128;
constexpr long long kOffDesc = 0;
constexpr long long kOffState = 256;
constexpr long long kOffJobs = 512;
// block sums of the grid preparation (at most 64 blocks of two doubles) and their counter
constexpr long long kOffRed = kOffJobs + kMaxJobs * (long long)sizeof(ToeplitzJob);
constexpr long long kOffRcnt = kOffRed + 64 * 16;
constexpr long long kOffGrid = kOffJobs + 65536LL * (long long)sizeof(ToeplitzJob);   // 256-aligned
constexpr long long kScratchBytes = kOffGrid + 2LL * 8LL * PRONY_STATIC_MAX_GRID;

static_assert(sizeof(ProbDesc) <= 256 && sizeof(ProbState) <= 256, "scratch header too small");
static_assert(kOffGrid % 256 == 0, "grid planes must stay 256-byte aligned");
static_assert(kOffRcnt + 16 <= kOffGrid, "reduction slots must fit below the grid planes");
static_assert(kScratchBytes == PRONY_STATIC_SCRATCH_BYTES, "scratch size must match the documented one");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Descriptor and job list written on the device (no host-to-device copy, no allocation).
__global__ void k_static_setup(ProbDesc desc, int tiles, int nks) {
  unsigned char* base = g_scratch;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *(ProbDesc*)(base + kOffDesc) = desc;
    *(int*)(base + kOffRcnt) = 0;
  }
  ToeplitzJob* jobs = (ToeplitzJob*)(base + kOffJobs);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < tiles * nks; q += gridDim.x * blockDim.x)
    jobs[q] = ToeplitzJob{0, q / nks, q % nks, nks};
}

}  // namespace

extern "C" int prony_toeplitz_mm_static(const prony_c128* grid_dev, int d, int n, const void* X_dev, int r, int L,
                                        int adjoint, void* Y_dev, void* stream) {
  if (!grid_dev || !X_dev || !Y_dev || d < 1 || d > PRONY_DMAX || n < 1 || r < 1 || r > PRONY_RMAX)
    return PRONY_EINVAL;
  if ((L != n + 1 && L != n + 2) || (adjoint && L != n + 1)) return PRONY_EINVAL;
  long long G = 2LL * n + 2, Gd = 1, N = 1, Next = 1;
  for (int l = 0; l < d; ++l) {
    Gd *= G;
    N *= n + 1;
    Next *= n + 2;
    if (Gd > PRONY_STATIC_MAX_GRID) {
      set_last_error("prony_toeplitz_mm_static: (2n+2)^d exceeds PRONY_STATIC_MAX_GRID samples of fixed scratch");
      return PRONY_EINVAL;
    }
  }
  if (r > N) {                                 // as prony_toeplitz_mm_dev: at most N columns
    set_last_error("prony_toeplitz_mm_static: r exceeds (n+1)^d");
    return PRONY_EINVAL;
  }
  // the device address of the array on the current device, looked up on every call
  void* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_scratch);
  if (e != cudaSuccess || !base) {
    set_last_error("prony_toeplitz_mm_static: cudaGetSymbolAddress of the scratch array failed");
    return PRONY_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long rows = (L == n + 2) ? Next : N;
  const int tiles = (int)((rows + 63) / 64);
  const int nks = 1;
  if ((long long)tiles * nks > kMaxJobs) return PRONY_EINVAL;

  ProbDesc desc{};
  desc.d = d;
  desc.n = n;
  desc.m = 1;
  desc.r0 = r;
  desc.N = (int)N;
  desc.Next = (int)Next;
  desc.G = (int)G;
  desc.Gd = (int)Gd;
  desc.grid = 0;
  desc.xoff = 0;
  desc.yoff = 0;
  desc.soff = 0;
  desc.ooff = 0;
  note_launch();
  k_static_setup<<<std::min(1024, (tiles * nks + 255) / 256), 256, 0, s>>>(desc, tiles, nks);

  unsigned char* b = (unsigned char*)base;
  Dev D{};
  D.P = (const ProbDesc*)(b + kOffDesc);
  D.st = (ProbState*)(b + kOffState);
  D.nprob = 1;
  D.maxN = (int)N;
  D.maxNext = (int)Next;
  D.maxGd = (int)Gd;
  D.maxR0 = r;
  D.maxM = 1;
  D.maxD = d;
  D.grid64 = (const double2*)grid_dev;
  D.gF = (float2*)(b + kOffGrid);
  D.gH = (float2*)(b + kOffGrid + 8LL * PRONY_STATIC_MAX_GRID);
  D.V = (float2*)X_dev;
  D.Y = (float2*)Y_dev;
  D.B2 = (float2*)Y_dev;
  D.small = nullptr;
  D.red = (char*)(b + kOffRed);
  D.red_stride = 64 * 16;
  D.rcnt = (int*)(b + kOffRcnt);
  // state (widths, flags) is rewritten by the first kernel; gF / gH are overwritten whole
  launch_prep(D, s);
  const ToeplitzJob* jobs = (const ToeplitzJob*)(b + kOffJobs);
  const int ext = (L == n + 2);
  launch_toeplitz(D, jobs, tiles * nks, adjoint, BUF_V, W_R0, ext ? BUF_Y : BUF_B2, ext, r, nullptr, nullptr, 0, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return PRONY_ECUDA;
  }
  return PRONY_OK;
}
