// decode.cuh -- decoder workspace and entry (see decode.cu).
#pragma once

#include "fic_internal.h"

namespace fic {

struct DecodeWs {
  DevBuf owner, x0, x1, ctl, delta;
  void release() {
    owner.release();
    x0.release();
    x1.release();
    ctl.release();
    delta.release();
  }
};

int decode_run(const fic_transform* d_codes, int64_t n_codes, int W, int H, int max_iters,
               double tol, DecodeWs& ws, uint8_t* d_out, int out_pitch, cudaStream_t st);

// o of every saved map in its stored form (o_bits bits over [-255, 255]);
// *n_codes is the device count of the level's maps.
int launch_quantize_o(fic_transform* codes, const int64_t* n_codes, int64_t cap, int o_bits,
                      cudaStream_t st);

}  // namespace fic

namespace fic {

// The decoder's kernels (decode.cu), also launched by the allocation-free
// entry point in decode_static.cu.
__global__ void k_owner_map(const fic_transform* __restrict__ codes, int64_t n_codes, int W,
                            int32_t* __restrict__ owner);
__global__ void k_fill(double* __restrict__ x, int64_t N, double v);
__global__ void k_decode_step(const fic_transform* __restrict__ codes,
                              const int32_t* __restrict__ owner, int W, int H,
                              const double* __restrict__ cur, double* __restrict__ nxt, int it,
                              double tol, int32_t* __restrict__ ctl,
                              unsigned long long* __restrict__ delta);
__global__ void k_decode_check(int it, double tol, int32_t* ctl, const unsigned long long* delta);
__global__ void k_decode_round(const double* __restrict__ a, const double* __restrict__ b,
                               const int32_t* __restrict__ ctl, int W, int H,
                               uint8_t* __restrict__ out, int pitch);

}  // namespace fic
