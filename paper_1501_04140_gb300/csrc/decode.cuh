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

}  // namespace fic
