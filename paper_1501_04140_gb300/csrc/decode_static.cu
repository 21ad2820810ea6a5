// decode_static.cu -- the decoder without any device allocation.
//
// fic_decode allocates its workspace (owner map, two FP64 iterates, control
// words) with cudaMalloc on first use.  Some callers cannot let a library do
// that: processes whose device memory is owned by another allocator (a
// framework's caching allocator or a pool sized once at start-up, where a
// foreign cudaMalloc fails or fragments the pool), and latency-bound loops in
// which cudaMalloc / cudaFree would synchronise the device.  For them,
// fic_decode_static runs the same decoder kernels on a workspace that is a
// file-scope __device__ array of this library, sized for images of up to
// FIC_DECODE_STATIC_MAX_PIXELS pixels and FIC_DECODE_STATIC_MAX_ITERS
// iterations.  The array is part of the library's device image: every GPU
// that loads the library holds it until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and keeps
// it for later calls.
#include <mutex>

#include "decode.cuh"

namespace fic {
namespace {

constexpr int64_t kMaxPix = FIC_DECODE_STATIC_MAX_PIXELS;
constexpr int kMaxIters = FIC_DECODE_STATIC_MAX_ITERS;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// workspace layout inside the array
constexpr size_t kOffOwner = 0;                                        // int32[kMaxPix]
constexpr size_t kOffX0 = align256(kOffOwner + sizeof(int32_t) * kMaxPix);  // double[kMaxPix]
constexpr size_t kOffX1 = align256(kOffX0 + sizeof(double) * kMaxPix);      // double[kMaxPix]
constexpr size_t kOffCtl = align256(kOffX1 + sizeof(double) * kMaxPix);     // int32[4]
constexpr size_t kOffBad = kOffCtl + 4 * sizeof(int32_t);                   // int32: bad codes
constexpr size_t kOffDelta = align256(kOffBad + sizeof(int32_t));           // u64[kMaxIters]
constexpr size_t kScratchBytes = align256(kOffDelta + sizeof(unsigned long long) * kMaxIters);

static __device__ __align__(256) unsigned char g_decode_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once).
int scratch_address(unsigned char** out) {
  int dev = -1;
  FIC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FIC_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_decode_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return e == cudaSuccess ? FIC_ECUDA : cuda_status(e);
    }
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return FIC_OK;
}

// Counts the codes whose blocks leave the W x H image or whose fields are out
// of range, so that no decoder kernel indexes outside its buffers.
__global__ void k_check_codes(const fic_transform* __restrict__ codes, int64_t n, int W, int H,
                              int32_t* __restrict__ bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const fic_transform t = codes[i];
    const int b = t.size;
    const bool size_ok = b == 2 || b == 4 || b == 8 || b == 16;
    const bool ok = size_ok && t.x >= 0 && t.y >= 0 && t.x <= W - b && t.y <= H - b &&
                    t.dom_x >= 0 && t.dom_y >= 0 && t.dom_x <= W - 2 * b &&
                    t.dom_y <= H - 2 * b && t.iso >= 0 && t.iso < 8 && t.s >= 0.0 && t.s <= 1.0;
    if (!ok) atomicAdd(bad, 1);
  }
}

}  // namespace
}  // namespace fic

using namespace fic;

extern "C" int fic_decode_static(const fic_transform* codes, int64_t n_codes, int width,
                                 int height, int max_iters, double tol, uint8_t* out,
                                 int out_pitch, void* stream, int* iters_done) {
  if (width <= 0 || height <= 0 || n_codes < 0 || (n_codes > 0 && !codes) || !out ||
      out_pitch < width || max_iters < 0)
    return FIC_EINVAL;
  const int64_t N = (int64_t)width * height;
  if (N > kMaxPix || max_iters > kMaxIters) return FIC_EINVAL;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  int32_t* owner = (int32_t*)(base + kOffOwner);
  double* x0 = (double*)(base + kOffX0);
  double* x1 = (double*)(base + kOffX1);
  int32_t* ctl = (int32_t*)(base + kOffCtl);
  int32_t* bad = (int32_t*)(base + kOffBad);
  unsigned long long* delta = (unsigned long long*)(base + kOffDelta);
  cudaStream_t st = (cudaStream_t)stream;

  // the previous call's contents stay in the array: reset what starts at zero
  FIC_CUDA_TRY(cudaMemsetAsync(ctl, 0, 4 * sizeof(int32_t) + sizeof(int32_t), st));
  FIC_CUDA_TRY(cudaMemsetAsync(delta, 0, sizeof(unsigned long long) * (max_iters > 0 ? max_iters : 1), st));
  if (n_codes > 0) {
    const int g = (int)(ceil_div64(n_codes, 256) < 1024 ? ceil_div64(n_codes, 256) : 1024);
    k_check_codes<<<g, 256, 0, st>>>(codes, n_codes, width, height, bad);
    FIC_CUDA_TRY(cudaGetLastError());
    int32_t nbad = 0;
    FIC_CUDA_TRY(cudaMemcpyAsync(&nbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    FIC_CUDA_TRY(cudaStreamSynchronize(st));
    if (nbad) return FIC_EINVAL;
  }

  // the same launches as fic_decode, on the array instead of allocated buffers
  FIC_CUDA_TRY(cudaMemsetAsync(owner, 0xff, sizeof(int32_t) * N, st));
  if (n_codes > 0)
    k_owner_map<<<(int)(n_codes < 65535 ? n_codes : 65535), 64, 0, st>>>(codes, n_codes, width,
                                                                         owner);
  const int threads = 256;
  const int grid = (int)(ceil_div64(N, threads) < 4096 ? ceil_div64(N, threads) : 4096);
  k_fill<<<grid, threads, 0, st>>>(x0, N, 128.0);
  for (int it = 0; it < max_iters; ++it) {
    const double* cur = (it & 1) ? x1 : x0;
    double* nxt = (it & 1) ? x0 : x1;
    k_decode_step<<<grid, threads, 0, st>>>(codes, owner, width, height, cur, nxt, it, tol, ctl,
                                            delta);
    k_decode_check<<<1, 1, 0, st>>>(it, tol, ctl, delta);
  }
  k_decode_round<<<grid, threads, 0, st>>>(x0, x1, ctl, width, height, out, out_pitch);
  FIC_CUDA_TRY(cudaGetLastError());
  int32_t done[2] = {0, 0};
  FIC_CUDA_TRY(cudaMemcpyAsync(done, ctl, sizeof(done), cudaMemcpyDeviceToHost, st));
  FIC_CUDA_TRY(cudaStreamSynchronize(st));
  if (iters_done) *iters_done = done[1];
  return FIC_OK;
}
