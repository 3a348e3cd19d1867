// pecc_noalloc.cu -- the feasibility check of one instance without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while its stream is being captured
// into a CUDA graph (an allocation there breaks or invalidates the capture), plug-ins whose
// host application owns every byte of device memory, and real-time loops where an
// allocation's latency or failure is not acceptable.  For them this entry point keeps its
// scratch (coordinates, cell counters, neighbor lists) in one fixed array in device memory,
// reserved when the library is loaded on a GPU and held by every GPU that loads the library
// until the process exits.  The caller passes the inputs and the outputs.
#include <mutex>

#include "pecc.h"
#include "pecc_internal.h"

namespace pecc {
namespace {

constexpr int kMaxN = PECC_NOALLOC_MAX_N;
constexpr int kMaxNc = 128;                      // max(16, ceil(2 sqrt(kMaxN)))
// Neighbor entries: the list capacity pecc_check_feasible builds with in a context created with the
// default nbr_capacity of 16 per circle, 2 (16 n + 64), taken per call and sized here for kMaxN.
__host__ __device__ constexpr int call_cap(int n) { return 2 * (16 * n + 64); }
constexpr int kCap = call_cap(kMaxN);
constexpr size_t kOffX = 0;                                   // double2[kMaxN]
constexpr size_t kOffXs = kOffX + sizeof(double2) * kMaxN;    // double2[kMaxN]
constexpr size_t kOffKey = kOffXs + sizeof(double2) * kMaxN;  // uint32[kMaxN]
constexpr size_t kOffOrd = kOffKey + 4 * (size_t)kMaxN;       // int32[kMaxN]
constexpr size_t kOffCells = kOffOrd + 4 * (size_t)kMaxN;     // int32[2 kMaxNc^2 + 2]
constexpr size_t kOffRp = kOffCells + 4 * (2 * (size_t)kMaxNc * kMaxNc + 2 + 2);  // int32[kMaxN + 1]
constexpr size_t kOffCol = kOffRp + 4 * ((size_t)kMaxN + 4);  // int32[kCap]
constexpr size_t kScratchBytes = kOffCol + 4 * (size_t)kCap;

// The scratch every call shares; its address is taken per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The array's device address per device, taken once by the first call on that device.  A
// cudaDeviceReset (or a lost context) on that device leaves this address stale.
std::mutex g_mu;
void *g_ptr[256];
bool g_ready[256];

__global__ void noalloc_feasible_kernel(unsigned char *scratch, const double *__restrict__ xy, int n, double R,
                                        double inv, int nc, double lc2, double tol, uint8_t *feasible,
                                        double *max_overlap) {
  const int cap = call_cap(n);
  __shared__ int32_t sh[40];
  __shared__ double red[32];
  double2 *x = (double2 *)(scratch + kOffX);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = make_double2(xy[2 * i], xy[2 * i + 1]);
  __syncthreads();
  const CellGrid G{R, inv, 0.f, 0.f, nc, false};
  int32_t *rp = (int32_t *)(scratch + kOffRp);
  int32_t *col = (int32_t *)(scratch + kOffCol);
  // the build zeroes the cell counters it uses and overwrites everything else it reads
  const int tot = cta_build_neighbors<double, int32_t>(
      x, n, G, lc2, (uint32_t *)(scratch + kOffKey), (int32_t *)(scratch + kOffOrd), (int32_t *)(scratch + kOffCells),
      (double2 *)(scratch + kOffXs), rp, col, cap, sh, nullptr, false);
  double m = 0.0;
  int bad = 0;
  if (tot <= cap) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double2 xi = x[i];
      bad |= !(isfinite(xi.x) && isfinite(xi.y));
      for (int t = rp[i]; t < rp[i + 1]; ++t) {
        const int j = col[t];
        if (j > i) m = fmax(m, pair_depth_exact(xi, x[j]));
      }
      m = fmax(m, wall_depth_exact(xi, R));
    }
  } else {
    bad = 1;
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
    if (bad) v = __longlong_as_double(0x7ff8000000000000ll);
    feasible[0] = (!bad && v <= tol) ? 1 : 0;
    max_overlap[0] = v;
  }
}

pecc_status err(pecc_status s, const char *msg) {
  set_global_error(msg);
  return s;
}

}  // namespace
}  // namespace pecc

using namespace pecc;

extern "C" pecc_status pecc_check_feasible_noalloc(const double *xy_dev, int32_t n, double R, double l_cut, double tol,
                                                   uint8_t *feasible_dev, double *max_overlap_dev, void *stream) {
  if (n < 0 || n > kMaxN) return err(PECC_ERR_ARG, "pecc_check_feasible_noalloc: n must be in 0..PECC_NOALLOC_MAX_N");
  if (!(R > 0.0) || !isfinite(R)) return err(PECC_ERR_ARG, "pecc_check_feasible_noalloc: R must be finite and > 0");
  if (!(l_cut > 2.0) || !isfinite(l_cut)) return err(PECC_ERR_ARG, "pecc_check_feasible_noalloc: l_cut must exceed 2");
  if (!feasible_dev || !max_overlap_dev || (n > 0 && !xy_dev))
    return err(PECC_ERR_ARG, "pecc_check_feasible_noalloc: NULL pointer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return err(PECC_ERR_CUDA, "pecc_check_feasible_noalloc: no current CUDA device");
  void *ptr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      // host code must not use g_scratch itself: it is a host-side stand-in for the device array
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
      if (e != cudaSuccess) return err(PECC_ERR_CUDA, cudaGetErrorString(e));
      g_ptr[dev] = ptr;
      g_ready[dev] = true;
    }
    ptr = g_ptr[dev];
  }
  double inv;
  int nc;
  host_cell_grid(R, l_cut, n, &inv, &nc);
  if (nc > kMaxNc) return err(PECC_ERR_ARG, "pecc_check_feasible_noalloc: cell grid over its maximum");
  noalloc_feasible_kernel<<<1, 256, 0, (cudaStream_t)stream>>>((unsigned char *)ptr, xy_dev, n, R, inv, nc,
                                                              l_cut * l_cut, tol, feasible_dev, max_overlap_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(PECC_ERR_CUDA, cudaGetErrorString(e));
  return PECC_OK;
}
