// decode.cu -- fixed-point decoder of the saved maps.
//
// The paper measures PSNR of decoded images but does not spell out the
// decoder; the reading used here is the usual one for fractal codes: start
// from a flat 128 image and apply every saved map to the previous iterate
// (Jacobi) in FP64,
//     x'(range pixel) = clamp_[0,255]( s * T_k(D(x))_pixel + o ),
// with D(x) the 2x2 mean of the domain block, until max |x' - x| < tol or
// max_iters iterations, then round half to even.  Each iteration's products
// and sums are formed in the same order as a plain sequential loop (no fused
// multiply-add) so that the iterate is reproducible.
#include <math.h>

#include "decode.cuh"

namespace fic {

// Stored form of o: rint((o + 255) / step) * step - 255 with
// step = 510 / (2^b - 1), clamped, each operation rounded on its own (no
// fused multiply-add), so that the value equals a plain sequential
// evaluation.
__global__ void k_quantize_o(fic_transform* __restrict__ codes, const int64_t* __restrict__ n_codes,
                             int o_bits) {
  const double levels = (double)((1LL << o_bits) - 1);
  const double step = __ddiv_rn(510.0, levels);
  const int64_t N = *n_codes;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double u = rint(__ddiv_rn(__dadd_rn(codes[i].o, 255.0), step));
    u = u < 0.0 ? 0.0 : (u > levels ? levels : u);
    codes[i].o = __dadd_rn(__dmul_rn(u, step), -255.0);
  }
}

int launch_quantize_o(fic_transform* codes, const int64_t* n_codes, int64_t cap, int o_bits,
                      cudaStream_t st) {
  int grid = (int)ceil_div64(cap > 0 ? cap : 1, 256);
  if (grid > 65535) grid = 65535;
  k_quantize_o<<<grid, 256, 0, st>>>(codes, n_codes, o_bits);
  return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

// Owner map: for each pixel, the code that writes it.
__global__ void k_owner_map(const fic_transform* __restrict__ codes, int64_t n_codes, int W,
                            int32_t* __restrict__ owner) {
  for (int64_t c = blockIdx.x; c < n_codes; c += gridDim.x) {
    const fic_transform t = codes[c];
    for (int e = threadIdx.x; e < t.size * t.size; e += blockDim.x) {
      const int i = e / t.size, j = e % t.size;
      owner[(int64_t)(t.y + i) * W + (t.x + j)] = (int32_t)c;
    }
  }
}

__global__ void k_fill(double* __restrict__ x, int64_t N, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// One Jacobi step.  ctl: [0] done flag, [1] iterations done; delta[it]
// collects max |x' - x| of iteration it (as ordered uint64 bits).
__global__ void k_decode_step(const fic_transform* __restrict__ codes,
                              const int32_t* __restrict__ owner, int W, int H,
                              const double* __restrict__ cur, double* __restrict__ nxt, int it,
                              double tol, int32_t* __restrict__ ctl,
                              unsigned long long* __restrict__ delta) {
  if (it > 0) {
    // iteration it - 1 decided whether to go on
    if (ctl[0]) return;
  }
  const int64_t N = (int64_t)W * H;
  double dmax = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = owner[p];
    if (c < 0) {  // not covered by any map: keep the value
      nxt[p] = cur[p];
      continue;
    }
    const fic_transform t = codes[c];
    const int y = (int)(p / W), x = (int)(p % W);
    const int i = y - t.y, j = x - t.x;
    int si, sj;
    iso_src(t.size, t.iso, i, j, &si, &sj);
    const double* d = cur + (int64_t)(t.dom_y + 2 * si) * W + (t.dom_x + 2 * sj);
    const double s = t.s;  // p / q, or Eq. 2's s of the exact-s mode
    double m = __dadd_rn(__dadd_rn(__dadd_rn(d[0], d[1]), d[W]), d[W + 1]);
    m = __dmul_rn(m, 0.25);
    double v = __dadd_rn(__dmul_rn(s, m), t.o);
    v = v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v);
    nxt[p] = v;
    const double a = fabs(v - cur[p]);
    dmax = a > dmax ? a : dmax;
  }
  // block max, then one atomic per block (non-negative doubles order as
  // their bit patterns)
  for (int o = 16; o > 0; o >>= 1) {
    const double other = __shfl_xor_sync(0xffffffffu, dmax, o);
    dmax = other > dmax ? other : dmax;
  }
  __shared__ double wmax[32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = dmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = wmax[w] > b ? wmax[w] : b;
    atomicMax(&delta[it], (unsigned long long)__double_as_longlong(b));
  }
}

// Runs after each step: records the count and stops once max |delta| < tol.
__global__ void k_decode_check(int it, double tol, int32_t* ctl,
                               const unsigned long long* delta) {
  if (ctl[0]) return;
  ctl[1] = it + 1;
  if (__longlong_as_double((long long)delta[it]) < tol) ctl[0] = 1;
}

__global__ void k_decode_round(const double* __restrict__ a, const double* __restrict__ b,
                               const int32_t* __restrict__ ctl, int W, int H,
                               uint8_t* __restrict__ out, int pitch) {
  // the result of iteration it (1-based count ctl[1]) sits in buffer it % 2
  const double* x = (ctl[1] & 1) ? b : a;
  const int64_t N = (int64_t)W * H;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    double v = rint(x[p]);
    v = v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v);
    out[(p / W) * pitch + (p % W)] = (uint8_t)v;
  }
}

// ---------------------------------------------------------------- one launch
// The whole fixed-point iteration in one cooperative launch: every block
// takes its pixels of each Jacobi step (the arithmetic of k_decode_step, in
// the same order), the blocks meet at a grid barrier, and all of them read
// the step's max |delta| and stop together once it is below tol (the test of
// k_decode_check); then they round the last iterate (k_decode_round).  So
// the result and the iteration count are those of the per-step launches,
// without a launch per step.  The iterates are read past L1 (__ldcg): other
// blocks wrote them.  The barrier waits are bounded (kWaitLimitNs): a block
// that gives up sets ctl[2] and leaves, and the host reports FIC_ETIMEOUT.

// Grid barrier over `nb` co-resident blocks: bar[0] counts arrivals, bar[1]
// is the generation.  False when the wait ran out.
__device__ inline bool grid_barrier(unsigned int* bar, unsigned int nb) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nb - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      for (unsigned int i = 0; *vgen == gen; ++i) {
        if ((i & 63) == 63) {
          unsigned long long t;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
          if (t - t0 > kWaitLimitNs) {
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(256)
k_decode_all(const fic_transform* __restrict__ codes, const int32_t* __restrict__ owner, int W,
             int H, double* x0, double* x1, int max_iters, double tol, int32_t* ctl,
             unsigned long long* delta, unsigned int* bar, uint8_t* __restrict__ out, int pitch) {
  const int64_t N = (int64_t)W * H;
  __shared__ double wmax[8];
  int done = 0;
  for (int it = 0; it < max_iters; ++it) {
    const double* cur = (it & 1) ? x1 : x0;
    double* nxt = (it & 1) ? x0 : x1;
    double dmax = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
      const int32_t c = owner[p];
      const double xc = __ldcg(cur + p);
      if (c < 0) {  // not covered by any map: keep the value
        nxt[p] = xc;
        continue;
      }
      const fic_transform t = codes[c];
      const int y = (int)(p / W), x = (int)(p % W);
      const int i = y - t.y, j = x - t.x;
      int si, sj;
      iso_src(t.size, t.iso, i, j, &si, &sj);
      const double* d = cur + (int64_t)(t.dom_y + 2 * si) * W + (t.dom_x + 2 * sj);
      const double s = t.s;
      double m = __dadd_rn(__dadd_rn(__dadd_rn(__ldcg(d), __ldcg(d + 1)), __ldcg(d + W)),
                           __ldcg(d + W + 1));
      m = __dmul_rn(m, 0.25);
      double v = __dadd_rn(__dmul_rn(s, m), t.o);
      v = v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v);
      nxt[p] = v;
      const double a = fabs(v - xc);
      dmax = a > dmax ? a : dmax;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, dmax, o);
      dmax = other > dmax ? other : dmax;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = dmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = wmax[w] > b ? wmax[w] : b;
      atomicMax(&delta[it], (unsigned long long)__double_as_longlong(b));
    }
    if (!grid_barrier(bar, gridDim.x)) {
      if (threadIdx.x == 0) atomicExch(&ctl[2], 1);
      return;
    }
    done = it + 1;
    const double dl = __longlong_as_double((long long)__ldcg((const unsigned long long*)&delta[it]));
    if (dl < tol) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl[0] = 1;
    ctl[1] = done;
  }
  const double* x = (done & 1) ? x1 : x0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    double v = rint(__ldcg(x + p));
    v = v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v);
    out[(p / W) * pitch + (p % W)] = (uint8_t)v;
  }
}

int decode_run(const fic_transform* d_codes, int64_t n_codes, int W, int H, int max_iters,
               double tol, DecodeWs& ws, uint8_t* d_out, int out_pitch, cudaStream_t st) {
  const int64_t N = (int64_t)W * H;
  if (ws.owner.reserve(sizeof(int32_t) * N) || ws.x0.reserve(sizeof(double) * N) ||
      ws.x1.reserve(sizeof(double) * N) || ws.ctl.reserve(sizeof(int32_t) * 8) ||
      ws.delta.reserve(sizeof(unsigned long long) * (max_iters > 0 ? max_iters : 1)))
    return FIC_ENOMEM;
  int32_t* owner = ws.owner.as<int32_t>();
  double* x0 = ws.x0.as<double>();
  double* x1 = ws.x1.as<double>();
  int32_t* ctl = ws.ctl.as<int32_t>();
  unsigned int* bar = (unsigned int*)(ctl + 4);  // ctl[0..3], then the barrier's two words
  unsigned long long* delta = ws.delta.as<unsigned long long>();
  FIC_CUDA_TRY(cudaMemsetAsync(owner, 0xff, sizeof(int32_t) * N, st));
  FIC_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(int32_t) * 8, st));
  FIC_CUDA_TRY(cudaMemsetAsync(delta, 0, sizeof(unsigned long long) * (max_iters > 0 ? max_iters : 1), st));
  if (n_codes > 0)
    k_owner_map<<<(int)(n_codes < 65535 ? n_codes : 65535), 64, 0, st>>>(d_codes, n_codes, W, owner);
  const int threads = 256;
  const int fgrid = (int)(ceil_div64(N, threads) < 4096 ? ceil_div64(N, threads) : 4096);
  k_fill<<<fgrid, threads, 0, st>>>(x0, N, 128.0);
  // as many blocks as fit at once on the device (a cooperative launch
  // refuses more), at most one pixel per thread
  int dev = 0, nsm = 0, per_sm = 0;
  FIC_CUDA_TRY(cudaGetDevice(&dev));
  FIC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decode_all, threads, 0));
  int64_t grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > ceil_div64(N, threads)) grid = ceil_div64(N, threads);
  if (grid < 1) grid = 1;
  unsigned int gridu = (unsigned int)grid;
  void* args[] = {(void*)&d_codes, (void*)&owner, (void*)&W,     (void*)&H,
                  (void*)&x0,      (void*)&x1,    (void*)&max_iters, (void*)&tol,
                  (void*)&ctl,     (void*)&delta, (void*)&bar,   (void*)&d_out,
                  (void*)&out_pitch};
  FIC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_decode_all, dim3(gridu), dim3(threads),
                                           args, 0, st));
  return FIC_OK;
}

}  // namespace fic
