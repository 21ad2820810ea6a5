// capi.cu -- the C ABI of include/fic.h: contexts, domain pools, single-level
// matching, the batched quadtree encoder and the decoder.
//
// The encoder runs level by level (Sec. 2: range sizes B0, B0/2, ...); every
// step is a kernel of this library and all counts that depend on the image
// (kept domains, ranges split) stay on the device, so one call enqueues the
// whole encode on the caller's stream without a host round trip.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "decode.cuh"
#include "fic_internal.h"
#include "level.cuh"
#include "scan.cuh"

using namespace fic;

// ---------------------------------------------------------------- buffers
int DevBuf::reserve(size_t want) {
  if (want == 0) want = 16;
  if (bytes >= want) return 0;
  release();
  if (cudaMalloc(&p, want) != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    cudaGetLastError();
    return FIC_ENOMEM;
  }
  bytes = want;
  return 0;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------- handles
struct fic_ctx {
  int device = 0;
  int nsm = 0;
  DevBuf dT;       // entropy-key increments, kKeyTableN + 1 int64
  int inject = 0;  // fault armed for the next tensor matcher launch (fic_debug_inject)
};

namespace {

// One quadtree level of a batch: pool, active ranges, plan, results.
struct LevelWs {
  int B = 0, n = 0, Kp = 0;
  PoolLevel pool;
  DevBuf img;                              // ImgDev per image (px, py of this level)
  int64_t cap = 0;                         // ranges capacity
  DevBuf rec, n_act, act_off, act_cnt, mom, gthr, apack, a32, res, acc, codes;
  DevBuf acc_cnt, rej_cnt, code_off;
  DevBuf item_off, chunks, meta, part;
  int64_t item_cap = 0, mt_cap = 0;
  int items_per_cta = 3;                   // the plan's work items per persistent CTA
  int groups_per_tile = 2;                 // tensor matcher, B <= 8: epilogue groups per tile
  bool tuned = false;                      // both chosen by timing (autotune)
  DevBuf scan_scr, total;
  void release_all() {
    DevBuf* all[] = {&pool.off,  &pool.img,   &pool.keys,   &pool.sd,    &pool.sq,     &pool.sel,
                     &pool.hist, &pool.kept,  &pool.bpack,  &pool.b32,   &pool.dom,    &pool.domf,
                     &pool.scan_scratch, &pool.total, &pool.slot_off, &pool.umax, &pool.run_off, &img, &rec, &n_act, &act_off,
                     &act_cnt,   &mom,        &gthr,        &apack,       &a32,        &res,         &acc,
                     &codes,     &acc_cnt,    &rej_cnt,     &code_off,   &item_off,    &chunks,
                     &meta,      &part,       &scan_scr,    &total};
    for (DevBuf* b : all) b->release();
  }
};

int kp_of(int B) { return B * B < 16 ? 16 : B * B; }

// Geometry of the pool of one level over the batch (host-known sizes).
void pool_geometry(PoolLevel& pl, const std::vector<fic_image>& ims, int B, int L) {
  const int ni = (int)ims.size();
  pl.B = B;
  pl.L = L;
  pl.n = B * B;
  pl.Kp = kp_of(B);
  pl.n_images = ni;
  pl.h_off.assign(ni + 1, 0);
  pl.h_slot_off.assign(ni + 1, 0);
  pl.h_run_off.assign(ni + 1, 0);
  pl.h_img.resize(ni);
  for (int i = 0; i < ni; ++i) {
    const int px = (ims[i].width - 2 * B) / L + 1, py = (ims[i].height - 2 * B) / L + 1;
    const int64_t P = (ims[i].width >= 2 * B && ims[i].height >= 2 * B) ? (int64_t)px * py : 0;
    pl.h_img[i] = ImgDev{nullptr, ims[i].width, ims[i].height, ims[i].pitch, px, py};
    pl.h_off[i + 1] = pl.h_off[i] + P;
    pl.h_run_off[i + 1] =
        pl.h_run_off[i] + (P > 0 ? (int64_t)py * pool_runs_per_row(px, B, L) : 0);
    pl.h_slot_off[i + 1] = pl.h_slot_off[i] + ceil_div64(P, kTileDoms) * kTileDoms;
  }
  pl.P_tot = pl.h_off[ni];
  pl.S_tot = pl.h_slot_off[ni];
}

int pool_alloc(PoolLevel& pl) {
  const int ni = pl.n_images;
  const int64_t P = pl.P_tot > 0 ? pl.P_tot : 1;
  const int64_t S = pl.S_tot + kTileDoms;  // one spare tile
  int rc = 0;
  rc |= pl.off.reserve(sizeof(int64_t) * (ni + 1));
  rc |= pl.slot_off.reserve(sizeof(int64_t) * (ni + 1));
  rc |= pl.run_off.reserve(sizeof(int64_t) * (ni + 1));
  rc |= pl.img.reserve(sizeof(ImgDev) * ni);
  rc |= pl.keys.reserve(sizeof(int64_t) * P);
  rc |= pl.sd.reserve(sizeof(int32_t) * P);
  rc |= pl.sq.reserve(sizeof(int32_t) * P);
  rc |= pl.sel.reserve(sizeof(SelState) * ni);
  rc |= pl.hist.reserve(sizeof(uint32_t) * kSelBins * ni);
  rc |= pl.kept.reserve(sizeof(int32_t) * S);
  rc |= pl.dom.reserve(sizeof(DomRec) * S);
  rc |= pl.domf.reserve(sizeof(float4) * S);
  rc |= pl.umax.reserve(16);
  if (pl.want_tc) rc |= pl.bpack.reserve((size_t)(S / kTileDoms) * tc_tile_bytes(pl.B));
  if (pl.want_f32) rc |= pl.b32.reserve(sizeof(float) * S * pl.n);
  rc |= pl.scan_scratch.reserve(sizeof(int32_t) * scan_scratch_blocks(P));
  rc |= pl.total.reserve(sizeof(int64_t) * 2);
  return rc ? FIC_ENOMEM : FIC_OK;
}

// The pool's size tables (fixed by the image sizes) ...
int pool_upload_sizes(PoolLevel& pl, cudaStream_t st) {
  FIC_CUDA_TRY(cudaMemcpyAsync(pl.off.p, pl.h_off.data(), sizeof(int64_t) * (pl.n_images + 1),
                               cudaMemcpyHostToDevice, st));
  FIC_CUDA_TRY(cudaMemcpyAsync(pl.slot_off.p, pl.h_slot_off.data(),
                               sizeof(int64_t) * (pl.n_images + 1), cudaMemcpyHostToDevice, st));
  FIC_CUDA_TRY(cudaMemcpyAsync(pl.run_off.p, pl.h_run_off.data(),
                               sizeof(int64_t) * (pl.n_images + 1), cudaMemcpyHostToDevice, st));
  return FIC_OK;
}

// ... and the image descriptors (device pointers of the images)
int pool_upload_images(PoolLevel& pl, const std::vector<const uint8_t*>& dev_pix, cudaStream_t st) {
  for (int i = 0; i < pl.n_images; ++i) pl.h_img[i].pix = dev_pix[i];
  FIC_CUDA_TRY(cudaMemcpyAsync(pl.img.p, pl.h_img.data(), sizeof(ImgDev) * pl.n_images,
                               cudaMemcpyHostToDevice, st));
  return FIC_OK;
}

int pool_upload(PoolLevel& pl, const std::vector<const uint8_t*>& dev_pix, cudaStream_t st) {
  int rc = pool_upload_sizes(pl, st);
  return rc ? rc : pool_upload_images(pl, dev_pix, st);
}

bool valid_image(const fic_image& im, int B0) {
  if (!im.pixels || im.width <= 0 || im.height <= 0 || im.pitch < im.width) return false;
  if (im.width % B0 || im.height % B0 || im.width < 2 * B0 || im.height < 2 * B0) return false;
  return true;
}

int check_params(const fic_params* p) {
  if (!p) return FIC_EINVAL;
  const int B0 = p->range_size0;
  if (B0 != 2 && B0 != 4 && B0 != 8 && B0 != 16) return FIC_EINVAL;
  if (p->n_levels < 1 || p->n_levels > 4 || (B0 >> (p->n_levels - 1)) < 2) return FIC_EINVAL;
  if (p->domain_step < 1) return FIC_EINVAL;
  if (p->s_mode != FIC_S_PREDEFINED && p->s_mode != FIC_S_GRID && p->s_mode != FIC_S_EXACT)
    return FIC_EINVAL;
  if (p->s_mode == FIC_S_GRID && (p->grid_samples < 2 || p->grid_samples > kMaxS))
    return FIC_EINVAL;
  if (!(p->entropy_percentile >= 0.0 && p->entropy_percentile <= 1.0)) return FIC_EINVAL;
  if (p->precision != FIC_PREC_TENSOR && p->precision != FIC_PREC_FP32) return FIC_EINVAL;
  if (!(p->rms_threshold >= 0.0)) return FIC_EINVAL;
  if (p->pool_size < 0) return FIC_EINVAL;
  // the exact-s search exists on the tensor path only
  if (p->s_mode == FIC_S_EXACT && p->precision != FIC_PREC_TENSOR) return FIC_EUNSUPPORTED;
  return FIC_OK;
}

// Device copies of host images (fic_image.host = 1) for the call's stream.
struct Staging {
  DevBuf buf;
  std::vector<const uint8_t*> dev_pix;
  int stage(const std::vector<fic_image>& ims, cudaStream_t st) {
    size_t total = 0;
    for (const auto& im : ims)
      if (im.host) total += ((size_t)im.width * im.height + 255) & ~(size_t)255;
    if (total && buf.reserve(total)) return FIC_ENOMEM;
    dev_pix.resize(ims.size());
    size_t off = 0;
    for (size_t i = 0; i < ims.size(); ++i) {
      const fic_image& im = ims[i];
      if (!im.host) {
        dev_pix[i] = im.pixels;
        continue;
      }
      uint8_t* d = buf.as<uint8_t>() + off;
      FIC_CUDA_TRY(cudaMemcpy2DAsync(d, im.width, im.pixels, im.pitch, im.width, im.height,
                                     cudaMemcpyHostToDevice, st));
      dev_pix[i] = d;
      off += ((size_t)im.width * im.height + 255) & ~(size_t)255;
    }
    return FIC_OK;
  }
  // images as the kernels see them (pitch = width for staged copies)
  std::vector<fic_image> device_view(const std::vector<fic_image>& ims) const {
    std::vector<fic_image> v = ims;
    for (size_t i = 0; i < v.size(); ++i)
      if (v[i].host) v[i].pitch = v[i].width;
    return v;
  }
};

__global__ void k_init_ranges(const int64_t* __restrict__ rng_off, int n_images,
                              const ImgDev* __restrict__ imgs, int B, RangeRec* __restrict__ rec,
                              int64_t* __restrict__ n_act, int64_t* __restrict__ act_off,
                              int64_t* __restrict__ act_cnt) {
  grid_dep_sync();
  const int64_t N = rng_off[n_images];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int im = find_segment(rng_off, n_images, g);
    const int64_t l = g - rng_off[im];
    const int nbx = imgs[im].W / B;
    rec[g] = RangeRec{im, (int)(l % nbx) * B, (int)(l / nbx) * B, -1};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *n_act = N;
    for (int i = 0; i < n_images; ++i) {
      act_off[i] = rng_off[i];
      act_cnt[i] = rng_off[i + 1] - rng_off[i];
    }
    act_off[n_images] = N;
  }
}

}  // namespace

// Encoder state and results of one fic_encode call.
struct fic_code {
  fic_ctx* ctx = nullptr;
  fic_params prm{};
  int n_images = 0, n_levels = 0;
  std::vector<fic_image> ims;      // as given (host flag kept)
  std::vector<fic_image> dims;     // as the kernels see them
  Staging staging;
  LevelWs lv[4];
  DevBuf rng_off;                  // level-0 range offsets
  DecodeWs dec;
  std::vector<int64_t> h_code_off[4];  // filled on first query
  std::vector<int64_t> h_rng_off;  // level-0 range offsets (host copy)
  // Read-back summary, one allocation: the code offsets of every level
  // (n_levels x (n_images + 1) int64; each level's code_off aliases its
  // slice) followed by the device status word of the last encode, so one
  // copy brings back everything a read of the codes needs first.
  DevBuf summary;
  DevBuf status;                   // alias of the summary's status word
  cudaStream_t st = nullptr;       // stream of the last encode
  // what the device holds of the host-side tables: the size tables are
  // uploaded once, the image descriptors when an image pointer changes
  bool sizes_up = false;
  std::vector<const uint8_t*> dev_pix_up;
  // replay of the device part of the encode (fic_encode_again)
  cudaGraphExec_t graph = nullptr;
  int64_t graph_kernels = 0;
  // optional per-level events around the matcher and the whole level
  bool profile = false;
  cudaEvent_t ev[4][4] = {};
  cudaEvent_t pev[4][2] = {};  // each level's pool build, on its side stream
  // the pools of levels 1.. depend on the images only: they are built on
  // side streams forked from the encode's stream, off the level chain
  cudaStream_t side[4] = {};
  cudaEvent_t fork_ev = nullptr, pool_ev[4] = {};
};

struct fic_pool {
  fic_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  DevBuf status;  // device status word (kStatus*)
  fic_params prm{};
  std::vector<fic_image> ims;
  Staging staging;
  PoolLevel pl;
};

struct fic_matches {
  fic_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  DevBuf status;  // device status word (kStatus*)
  int64_t n = 0;
  LevelWs ws;
};

// ---------------------------------------------------------------- level driver
namespace {

// An event record that survives stream capture: inside a capture a plain
// record only orders the captured work, an external record becomes an
// event-record node of the graph that is recorded at every replay.
cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return cudaGetLastError();
  if (cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  return cudaEventRecord(e, st);
}

int level_alloc(fic_ctx* ctx, LevelWs& w, const std::vector<fic_image>& ims, int B, int64_t cap,
                const fic_params& prm) {
  const int ni = (int)ims.size();
  w.B = B;
  w.n = B * B;
  w.Kp = kp_of(B);
  w.cap = cap;
  // default shape (measured on a 512 x 512 encode): one epilogue group per
  // tile (16 ranges per warp visit) at B <= 4, two at B = 8
  w.groups_per_tile = 2;
  const int64_t C = cap + kTileRanges;  // one spare M tile
  const bool tc = prm.precision == FIC_PREC_TENSOR;
  int rc = 0;
  rc |= w.rec.reserve(sizeof(RangeRec) * C);
  rc |= w.n_act.reserve(sizeof(int64_t) * 2);
  rc |= w.act_off.reserve(sizeof(int64_t) * (ni + 1));
  rc |= w.act_cnt.reserve(sizeof(int64_t) * ni);
  rc |= w.mom.reserve(sizeof(RangeMom) * C);
  rc |= w.gthr.reserve(sizeof(uint32_t) * C);
  if (tc) rc |= w.apack.reserve(sizeof(uint16_t) * C * 8 * w.Kp);
  else rc |= w.a32.reserve(sizeof(float) * C * 8 * w.n);
  rc |= w.res.reserve(sizeof(fic_transform) * C);
  rc |= w.acc.reserve(C);
  rc |= w.codes.reserve(sizeof(fic_transform) * C);
  rc |= w.acc_cnt.reserve(sizeof(int32_t) * ni);
  rc |= w.rej_cnt.reserve(sizeof(int32_t) * ni);
  rc |= w.code_off.reserve(sizeof(int64_t) * (ni + 1));
  rc |= w.item_off.reserve(sizeof(int64_t) * (ni + 1));
  rc |= w.chunks.reserve(sizeof(int32_t) * ni);
  rc |= w.meta.reserve(sizeof(PlanMeta));
  int64_t mt = 0;
  for (int i = 0; i < ni; ++i) {
    const int64_t ri = (int64_t)(ims[i].width / B) * (ims[i].height / B);
    mt += ceil_div64(ri < cap ? ri : cap, kTileRanges);
  }
  w.mt_cap = mt;
  w.item_cap = mt + 8 * (int64_t)ctx->nsm;
  rc |= w.part.reserve(sizeof(Cand) * w.item_cap * kTileRows);
  rc |= w.scan_scr.reserve(sizeof(int32_t) * scan_scratch_blocks(C));
  rc |= w.total.reserve(sizeof(int64_t) * 2);
  w.pool.want_tc = tc;
  w.pool.want_f32 = !tc;
  make_sset(prm.s_mode, prm.grid_samples, B, &w.pool.sset);
  w.pool.pct = prm.entropy_percentile;
  w.pool.top_k = prm.pool_size;
  return rc ? FIC_ENOMEM : FIC_OK;
}

// The work plan of one level: its pool's kept counts and its active ranges
// give the work items; with_split also zeroes the split counters per tile.
PlanArgs plan_args(const fic_ctx* ctx, LevelWs& w, int items_per_cta, bool with_split) {
  PlanArgs p{};
  p.n_images = w.pool.n_images;
  p.sel = w.pool.sel.as<SelState>();
  p.target_items = items_per_cta * ctx->nsm;
  p.item_cap = w.item_cap;
  p.mt_cap = w.mt_cap;
  p.meta = w.meta.as<PlanMeta>();
  p.item_off = w.item_off.as<int64_t>();
  p.chunks = w.chunks.as<int32_t>();
  p.acc_cnt = w.acc_cnt.as<int32_t>();
  p.rej_cnt = w.rej_cnt.as<int32_t>();
  p.tile_acc = with_split ? w.scan_scr.as<int32_t>() : nullptr;
  p.n_tiles = (int)ceil_div64(w.cap > 0 ? w.cap : 1, kScanTile);
  return p;
}

// Matching of the active ranges of one level against the level's pool,
// then the exact map of every range (res).
// With split >= 0 the reducer also takes the level's split decision (split =
// 1 on the last level, which accepts every range).  A pool built on another
// stream joins through pool_ready, after the range operand and before the
// plan, the first step that reads the pool.  planned: the previous level's
// split kernel has already written this level's plan (for the level's
// current schedule), so only a re-tune plans again here.
int level_match(fic_ctx* ctx, LevelWs& w, const fic_params& prm, int level, uint32_t* status,
                cudaStream_t st, cudaEvent_t* ev = nullptr, int split = -1,
                cudaEvent_t pool_ready = nullptr, bool planned = false) {
  PoolLevel& pl = w.pool;
  const int ni = pl.n_images;
  const bool tc = prm.precision == FIC_PREC_TENSOR;
  const int grid = ctx->nsm;
  int32_t* tile_acc = split >= 0 ? w.scan_scr.as<int32_t>() : nullptr;
  // range operand (also resets the ranges' shared thresholds) and the plan
  auto pack_plan = [&](int items_per_cta, bool plan) -> int {
    int rc = launch_range_pack(w.B, pl.img.as<ImgDev>(), w.rec.as<RangeRec>(),
                               w.n_act.as<int64_t>(), w.cap, w.Kp, w.mom.as<RangeMom>(),
                               w.gthr.as<uint32_t>(), tc ? w.apack.as<uint16_t>() : nullptr,
                               tc ? nullptr : w.a32.as<float>(), ctx->nsm, st);
    if (rc || !plan) return rc;
    if (pool_ready) FIC_CUDA_TRY(cudaStreamWaitEvent(st, pool_ready, 0));
    const cudaError_t e =
        launch_dep(k_plan, dim3(1), dim3(256), 0, st, plan_args(ctx, w, items_per_cta, split >= 0),
                   (const int64_t*)w.act_off.as<int64_t>(), (const int64_t*)w.act_cnt.as<int64_t>());
    return e == cudaSuccess ? FIC_OK : FIC_ECUDA;
  };
  MatchArgs a{};
  a.B = w.B;
  a.n = w.n;
  a.Kp = w.Kp;
  a.n_images = ni;
  a.S = pl.sset;
  a.delta = screening_delta(w.B, pl.sset);
  a.mom = w.mom.as<RangeMom>();
  a.apack = w.apack.as<uint16_t>();
  a.a32 = w.a32.as<float>();
  a.bpack = pl.bpack.as<uint16_t>();
  a.b32 = pl.b32.as<float>();
  a.dom = pl.dom.as<DomRec>();
  a.domf = pl.domf.as<float>();
  a.gthr = w.gthr.as<uint32_t>();
  a.umax = pl.umax.as<float>();
  a.act_off = w.act_off.as<int64_t>();
  a.act_cnt = w.act_cnt.as<int64_t>();
  a.pool_off = pl.slot_off.as<int64_t>();
  a.sel = pl.sel.as<SelState>();
  a.item_off = w.item_off.as<int64_t>();
  a.chunks = w.chunks.as<int32_t>();
  a.meta = w.meta.as<PlanMeta>();
  a.pm = PosMoments{pl.sd.as<int32_t>(), pl.sq.as<int32_t>(), pl.off.as<int64_t>()};
  a.part = w.part.as<Cand>();
  a.groups_per_tile = w.groups_per_tile;
  a.status = status;
  // a fault armed by fic_debug_inject goes to the next tensor launch only
  auto match = [&]() {
    if (!tc) return launch_match_f32(a, grid, st);
    a.inject = ctx->inject;
    ctx->inject = 0;
    return launch_match_tc(a, grid, st);
  };

  // autotune: on the level's first eager run, time the matcher over a grid
  // of schedules -- work items per persistent CTA, and at B <= 8 on the
  // tensor path the epilogue groups per tile (two groups with 8 ranges per
  // warp visit, or one with 16) -- each candidate from freshly reset
  // thresholds, one untimed launch and then the median of kTrials timed
  // ones, and keep the fastest for the level's later encodes and the
  // captured graph
  if (prm.autotune && !w.tuned) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    FIC_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      static const int kItems[] = {2, 3, 4, 6, 8};
      constexpr int kTrials = 5;
      const int n_groups = (tc && w.B <= 8) ? 2 : 1;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      int rc = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess
                   ? FIC_OK
                   : FIC_ECUDA;
      float best = INFINITY;
      int best_items = w.items_per_cta, best_groups = w.groups_per_tile;
      for (int gi = 0; !rc && gi < n_groups; ++gi) {
        a.groups_per_tile = n_groups == 1 ? w.groups_per_tile : 2 - gi;
        for (int cand : kItems) {
          if (rc) break;
          float ms[kTrials];
          // one untimed launch: a kernel's first launch carries one-time
          // costs (module loading) that would count against the candidate
          for (int t = -1; !rc && t < kTrials; ++t) {
            if ((rc = pack_plan(cand, true))) break;
            if (t < 0) {
              rc = match();
              continue;
            }
            if (cudaEventRecord(e0, st) != cudaSuccess || (rc = match()) ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms[t], e0, e1) != cudaSuccess)
              rc = rc ? rc : FIC_ECUDA;
          }
          if (rc) break;
          std::sort(ms, ms + kTrials);
          if (ms[kTrials / 2] < best) {
            best = ms[kTrials / 2];
            best_items = cand;
            best_groups = a.groups_per_tile;
          }
        }
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (rc) return rc;
      w.items_per_cta = best_items;
      w.groups_per_tile = best_groups;
      a.groups_per_tile = best_groups;
      w.tuned = true;
      planned = false;  // the candidates overwrote the plan
    }
  }

  int rc = pack_plan(w.items_per_cta, !planned);
  if (rc) return rc;
  if (ev) FIC_CUDA_TRY(record_event(ev[1], st));
  if ((rc = match())) return rc;
  if (ev) FIC_CUDA_TRY(record_event(ev[2], st));
  return launch_reduce_final(w.B, pl.img.as<ImgDev>(), w.rec.as<RangeRec>(), w.n_act.as<int64_t>(),
                             w.cap, w.act_off.as<int64_t>(), pl.slot_off.as<int64_t>(), ni, pl.L,
                             pl.sel.as<SelState>(), w.item_off.as<int64_t>(),
                             w.chunks.as<int32_t>(), w.part.as<Cand>(), tc ? 1 : 8, pl.sset, level,
                             w.meta.as<PlanMeta>(), status,
                             w.res.as<fic_transform>(), prm.rms_threshold, split > 0 ? 1 : 0,
                             split >= 0 ? w.acc.as<uint8_t>() : nullptr, w.acc_cnt.as<int32_t>(),
                             w.rej_cnt.as<int32_t>(), tile_acc, a.pm,
                             tc ? w.mom.as<RangeMom>() : nullptr, ctx->nsm, st);
}

int64_t ranges_at(const std::vector<fic_image>& ims, int B) {
  int64_t s = 0;
  for (const auto& im : ims) s += (int64_t)(im.width / B) * (im.height / B);
  return s;
}

// Host -> device part of an encode: staging of host images, the image
// descriptors of every level and the level-0 range offsets.  Everything
// after it (encode_device) reads device memory only, so it can be captured
// into a CUDA graph and replayed.
int encode_upload(fic_code* c, cudaStream_t st) {
  const int ni = c->n_images;
  int rc = c->staging.stage(c->ims, st);
  if (rc) return rc;
  if (!c->sizes_up) {
    const int B0 = c->prm.range_size0;
    std::vector<int64_t>& roff = c->h_rng_off;
    roff.assign(ni + 1, 0);
    for (int i = 0; i < ni; ++i)
      roff[i + 1] = roff[i] + (int64_t)(c->dims[i].width / B0) * (c->dims[i].height / B0);
    if (c->rng_off.reserve(sizeof(int64_t) * (ni + 1))) return FIC_ENOMEM;
    FIC_CUDA_TRY(cudaMemcpyAsync(c->rng_off.p, roff.data(), sizeof(int64_t) * (ni + 1),
                                 cudaMemcpyHostToDevice, st));
    for (int l = 0; l < c->n_levels; ++l)
      if ((rc = pool_upload_sizes(c->lv[l].pool, st))) return rc;
    c->sizes_up = true;
  }
  if (c->dev_pix_up != c->staging.dev_pix) {
    for (int l = 0; l < c->n_levels; ++l)
      if ((rc = pool_upload_images(c->lv[l].pool, c->staging.dev_pix, st))) return rc;
    c->dev_pix_up = c->staging.dev_pix;
  }
  return FIC_OK;
}

int encode_device(fic_code* c, cudaStream_t st) {
  fic_ctx* ctx = c->ctx;
  const fic_params& prm = c->prm;
  const int ni = c->n_images;
  const int B0 = prm.range_size0;
  int rc = FIC_OK;
  // a fresh status for this encode (also a node of the captured graph, so
  // every replay starts clear)
  FIC_CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 16, st));
  // fork: every level's pool on its own side stream; level 0 joins its pool
  // before its plan, so level 0's ranges are set up meanwhile, and level
  // l + 1's pool joins before level l's split, which plans level l + 1
  FIC_CUDA_TRY(cudaEventRecord(c->fork_ev, st));
  for (int l = 0; l < c->n_levels; ++l) {
    FIC_CUDA_TRY(cudaStreamWaitEvent(c->side[l], c->fork_ev, 0));
    if (c->profile) FIC_CUDA_TRY(record_event(c->pev[l][0], c->side[l]));
    if ((rc = pool_build(c->lv[l].pool, ctx->dT.as<int64_t>(), c->side[l]))) return rc;
    if (c->profile) FIC_CUDA_TRY(record_event(c->pev[l][1], c->side[l]));
    FIC_CUDA_TRY(cudaEventRecord(c->pool_ev[l], c->side[l]));
  }
  for (int l = 0; l < c->n_levels; ++l) {
    LevelWs& w = c->lv[l];
    PoolLevel& pl = w.pool;
    if (c->profile) FIC_CUDA_TRY(record_event(c->ev[l][0], st));
    if (l == 0) {
      const int64_t nr = c->h_rng_off[ni];
      const int grid = (int)std::min<int64_t>(65535, ceil_div64(std::max<int64_t>(nr, 1), 256));
      FIC_CUDA_TRY(launch_dep(k_init_ranges, dim3(grid), dim3(256), 0, st,
                              (const int64_t*)c->rng_off.as<int64_t>(), ni,
                              (const ImgDev*)pl.img.as<ImgDev>(), B0, w.rec.as<RangeRec>(),
                              w.n_act.as<int64_t>(), w.act_off.as<int64_t>(),
                              w.act_cnt.as<int64_t>()));
    }
    const bool last = (l == c->n_levels - 1);
    if ((rc = level_match(ctx, w, prm, l, c->status.as<uint32_t>(), st,
                          c->profile ? c->ev[l] : nullptr, last ? 1 : 0,
                          l == 0 ? c->pool_ev[0] : nullptr, l > 0)))
      return rc;
    LevelWs* nx = last ? nullptr : &c->lv[l + 1];
    PlanArgs np{};
    if (nx) {
      FIC_CUDA_TRY(cudaStreamWaitEvent(st, c->pool_ev[l + 1], 0));
      np = plan_args(ctx, *nx, nx->items_per_cta, true);
    }
    rc = launch_split(w.res.as<fic_transform>(), w.rec.as<RangeRec>(), w.n_act.as<int64_t>(), w.cap,
                      w.B, ni, w.acc.as<uint8_t>(),
                      w.acc_cnt.as<int32_t>(), w.rej_cnt.as<int32_t>(), w.code_off.as<int64_t>(),
                      w.codes.as<fic_transform>(), nx ? nx->rec.as<RangeRec>() : nullptr,
                      nx ? nx->act_off.as<int64_t>() : nullptr,
                      nx ? nx->act_cnt.as<int64_t>() : nullptr,
                      nx ? nx->n_act.as<int64_t>() : nullptr,
                      w.scan_scr.as<int32_t>(), w.total.as<int64_t>(), nx ? &np : nullptr, st);
    if (rc) return rc;
    if (c->profile) FIC_CUDA_TRY(record_event(c->ev[l][3], st));
  }
  FIC_CUDA_TRY(cudaGetLastError());
  return FIC_OK;
}

int encode_enqueue(fic_code* c, cudaStream_t st) {
  c->st = st;
  int rc = encode_upload(c, st);
  if (!rc) rc = encode_device(c, st);
  return rc;
}

// Capture encode_device once into a graph (on a non-default stream) and
// replay it; the kernels it holds are counted for the caller.
int encode_graph(fic_code* c, cudaStream_t st) {
  c->st = st;
  int rc = encode_upload(c, st);
  if (rc) return rc;
  if (!c->graph) {
    cudaGraph_t g = nullptr;
    FIC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    rc = encode_device(c, st);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc ? rc : FIC_ECUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int64_t k = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    c->graph_kernels = k;
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return FIC_ECUDA;
    }
  }
  FIC_CUDA_TRY(cudaGraphLaunch(c->graph, st));
  return FIC_OK;
}

// Waits for `st` and reports the device status word of a handle.
int sync_and_status(const DevBuf& status, cudaStream_t st) {
  FIC_CUDA_TRY(cudaStreamSynchronize(st));
  uint32_t s = 0;
  FIC_CUDA_TRY(cudaMemcpy(&s, status.p, sizeof(s), cudaMemcpyDeviceToHost));
  if (s & kStatusTimeout) return FIC_ETIMEOUT;
  if (s & kStatusOverflow) return FIC_ERANGE;
  return FIC_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" {

const char* fic_status_string(int s) {
  switch (s) {
    case FIC_OK: return "FIC_OK";
    case FIC_EINVAL: return "FIC_EINVAL: invalid argument";
    case FIC_ENOMEM: return "FIC_ENOMEM: allocation failed";
    case FIC_ECUDA: return "FIC_ECUDA: CUDA call failed";
    case FIC_ETIMEOUT: return "FIC_ETIMEOUT: bounded device wait expired";
    case FIC_EUNSUPPORTED: return "FIC_EUNSUPPORTED: device is not sm_103";
    case FIC_ERANGE: return "FIC_ERANGE: capacity too small";
    default: return "unknown status";
  }
}

int fic_version(void) { return FIC_VERSION; }

int fic_default_params(fic_params* out) {
  if (!out) return FIC_EINVAL;
  fic_params p{};
  p.n_levels = 4;
  p.range_size0 = 16;
  p.domain_step = 2;
  p.rms_threshold = 8.0;
  p.single_level = 0;
  p.s_mode = FIC_S_PREDEFINED;
  p.grid_samples = 16;
  p.entropy_percentile = 0.5;
  p.precision = FIC_PREC_TENSOR;
  p.autotune = 0;
  p.pool_size = 0;
  *out = p;
  return FIC_OK;
}

int fic_create(fic_ctx** out, int device) {
  if (!out) return FIC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FIC_ECUDA;
  }
  cudaDeviceProp prop{};
  FIC_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) return FIC_EUNSUPPORTED;
  FIC_CUDA_TRY(cudaSetDevice(device));
  fic_ctx* c = new (std::nothrow) fic_ctx();
  if (!c) return FIC_ENOMEM;
  c->device = device;
  c->nsm = prop.multiProcessorCount;
  if (match_tc_prepare() != FIC_OK || pool_prepare() != FIC_OK) {
    delete c;
    return FIC_ECUDA;
  }
  std::vector<int64_t> dT(kKeyTableN + 1);
  host_key_table(dT.data(), kKeyTableN);
  if (c->dT.reserve(sizeof(int64_t) * dT.size())) {
    c->dT.release();
    delete c;
    return FIC_ENOMEM;
  }
  if (cudaMemcpy(c->dT.p, dT.data(), sizeof(int64_t) * dT.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    c->dT.release();
    delete c;
    return FIC_ECUDA;
  }
  *out = c;
  return FIC_OK;
}

int fic_destroy(fic_ctx* c) {
  if (!c) return FIC_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->dT.release();
  delete c;
  return FIC_OK;
}

int fic_debug_inject(fic_ctx* c, int fault) {
  if (!c || (fault != FIC_FAULT_NONE && fault != FIC_FAULT_DROP_TILE_COPY)) return FIC_EINVAL;
  c->inject = fault;
  return FIC_OK;
}

// ------------------------------------------------------------ pools
int fic_build_domain_pool(fic_ctx* ctx, const fic_image* img, int range_size,
                          const fic_params* params, void* stream, fic_pool** out) {
  if (!ctx || !img || !out || !params) return FIC_EINVAL;
  if (const int pc = check_params(params)) return pc;
  *out = nullptr;
  if (range_size != 2 && range_size != 4 && range_size != 8 && range_size != 16) return FIC_EINVAL;
  if (!valid_image(*img, range_size)) return FIC_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  fic_pool* p = new (std::nothrow) fic_pool();
  if (!p) return FIC_ENOMEM;
  p->ctx = ctx;
  p->st = st;
  p->prm = *params;
  p->ims = {*img};
  int rc = p->status.reserve(16);
  if (!rc && cudaMemsetAsync(p->status.p, 0, 16, st) != cudaSuccess) rc = FIC_ECUDA;
  if (!rc) rc = p->staging.stage(p->ims, st);
  if (!rc) {
    std::vector<fic_image> dv = p->staging.device_view(p->ims);
    pool_geometry(p->pl, dv, range_size, params->domain_step);
    p->pl.nsm = ctx->nsm;
    p->pl.want_tc = params->precision == FIC_PREC_TENSOR;
    p->pl.want_f32 = !p->pl.want_tc;
    make_sset(params->s_mode, params->grid_samples, range_size, &p->pl.sset);
    p->pl.pct = params->entropy_percentile;
    p->pl.top_k = params->pool_size;
    rc = pool_alloc(p->pl);
    if (!rc) rc = pool_upload(p->pl, p->staging.dev_pix, st);
    if (!rc) rc = pool_build(p->pl, ctx->dT.as<int64_t>(), st);
  }
  if (rc) {
    fic_pool_free(p);
    return rc;
  }
  *out = p;
  return FIC_OK;
}

int fic_pool_info(const fic_pool* p, fic_pool_info_t* out) {
  if (!p || !out) return FIC_EINVAL;
  int rc = sync_and_status(p->status, p->st);
  if (rc) return rc;
  SelState s{};
  FIC_CUDA_TRY(cudaMemcpy(&s, p->pl.sel.p, sizeof(s), cudaMemcpyDeviceToHost));
  out->size = p->pl.B;
  out->step = p->pl.L;
  out->px = p->pl.h_img[0].px;
  out->py = p->pl.h_img[0].py;
  out->pool_size = (int32_t)p->pl.P_tot;
  out->n_kept = s.nkept;
  out->fallback = s.fallback;
  out->reserved = 0;
  out->thr_key = s.thr;
  return FIC_OK;
}

int fic_pool_copy(const fic_pool* p, int field, void* host_dst, size_t bytes) {
  if (!p || !host_dst) return FIC_EINVAL;
  int rc = sync_and_status(p->status, p->st);
  if (rc) return rc;
  SelState s{};
  FIC_CUDA_TRY(cudaMemcpy(&s, p->pl.sel.p, sizeof(s), cudaMemcpyDeviceToHost));
  const size_t nk = (size_t)s.nkept;
  const int64_t slot0 = p->pl.h_slot_off[0];
  switch (field) {
    case FIC_POOL_KEYS: {
      const size_t need = sizeof(int64_t) * (size_t)p->pl.P_tot;
      if (bytes < need) return FIC_ERANGE;
      FIC_CUDA_TRY(cudaMemcpy(host_dst, p->pl.keys.p, need, cudaMemcpyDeviceToHost));
      return FIC_OK;
    }
    case FIC_POOL_KEPT: {
      if (bytes < sizeof(int32_t) * nk) return FIC_ERANGE;
      FIC_CUDA_TRY(cudaMemcpy(host_dst, p->pl.kept.as<int32_t>() + slot0, sizeof(int32_t) * nk,
                              cudaMemcpyDeviceToHost));
      return FIC_OK;
    }
    case FIC_POOL_SUMS:
    case FIC_POOL_SQSUMS: {
      if (bytes < sizeof(int64_t) * nk) return FIC_ERANGE;
      std::vector<int32_t> kept(nk), v((size_t)p->pl.P_tot);
      FIC_CUDA_TRY(cudaMemcpy(kept.data(), p->pl.kept.as<int32_t>() + slot0, sizeof(int32_t) * nk,
                              cudaMemcpyDeviceToHost));
      FIC_CUDA_TRY(cudaMemcpy(v.data(), field == FIC_POOL_SUMS ? p->pl.sd.p : p->pl.sq.p,
                              sizeof(int32_t) * v.size(), cudaMemcpyDeviceToHost));
      int64_t* o = (int64_t*)host_dst;
      for (size_t j = 0; j < nk; ++j) o[j] = v[(size_t)kept[j]];
      return FIC_OK;
    }
    default: return FIC_EINVAL;
  }
}

void fic_pool_free(fic_pool* p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  PoolLevel& pl = p->pl;
  DevBuf* all[] = {&pl.off,  &pl.slot_off, &pl.img, &pl.keys, &pl.sd,   &pl.sq,   &pl.sel,
                   &pl.hist, &pl.kept,     &pl.bpack, &pl.b32, &pl.dom, &pl.domf, &pl.scan_scratch,
                   &pl.total, &pl.umax, &pl.run_off};
  for (DevBuf* b : all) b->release();
  p->staging.buf.release();
  p->status.release();
  delete p;
}

// ------------------------------------------------------------ one level
int fic_match_level(fic_ctx* ctx, const fic_image* img, const fic_pool* pool,
                    const int32_t* range_xy, int n_ranges, const fic_params* params, void* stream,
                    fic_matches** out) {
  if (!ctx || !img || !pool || !out || !params || n_ranges < 0) return FIC_EINVAL;
  if (const int pc = check_params(params)) return pc;
  if (n_ranges > 0 && !range_xy) return FIC_EINVAL;
  *out = nullptr;
  const int B = pool->pl.B;
  if (img->width != pool->ims[0].width || img->height != pool->ims[0].height) return FIC_EINVAL;
  if ((params->precision == FIC_PREC_TENSOR) != pool->pl.want_tc) return FIC_EINVAL;
  // the pool's per-domain scoring records were built for its S set
  if (params->s_mode != pool->prm.s_mode ||
      (params->s_mode == FIC_S_GRID && params->grid_samples != pool->prm.grid_samples))
    return FIC_EINVAL;
  for (int r = 0; r < n_ranges; ++r) {
    const int x = range_xy[2 * r], y = range_xy[2 * r + 1];
    if (x < 0 || y < 0 || x + B > img->width || y + B > img->height) return FIC_EINVAL;
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  fic_matches* m = new (std::nothrow) fic_matches();
  if (!m) return FIC_ENOMEM;
  m->ctx = ctx;
  m->st = st;
  m->n = n_ranges;
  std::vector<fic_image> ims = pool->staging.device_view(pool->ims);
  LevelWs& w = m->ws;
  int rc = level_alloc(ctx, w, ims, B, std::max(n_ranges, 1), *params);
  if (!rc) rc = m->status.reserve(16);
  if (!rc && cudaMemsetAsync(m->status.p, 0, 16, st) != cudaSuccess) rc = FIC_ECUDA;
  if (!rc) {
    // the level works on the pool's buffers; share them without copying
    w.pool = PoolLevel();
    PoolLevel& src = const_cast<fic_pool*>(pool)->pl;
    w.pool.B = src.B; w.pool.L = src.L; w.pool.n = src.n; w.pool.Kp = src.Kp;
    w.pool.n_images = 1; w.pool.P_tot = src.P_tot; w.pool.S_tot = src.S_tot;
    w.pool.h_off = src.h_off; w.pool.h_slot_off = src.h_slot_off; w.pool.h_img = src.h_img;
    w.pool.want_tc = src.want_tc; w.pool.want_f32 = src.want_f32;
    make_sset(params->s_mode, params->grid_samples, B, &w.pool.sset);
    w.pool.pct = src.pct;
    w.pool.top_k = src.top_k;
    // borrowed pointers (not released by this handle)
    w.pool.img = src.img; w.pool.sel = src.sel; w.pool.slot_off = src.slot_off;
    w.pool.bpack = src.bpack; w.pool.b32 = src.b32; w.pool.dom = src.dom;
    w.pool.domf = src.domf;
    w.pool.umax = src.umax;
    w.pool.sd = src.sd; w.pool.sq = src.sq; w.pool.off = src.off;  // per-position sums
    std::vector<RangeRec> rec(n_ranges);
    for (int r = 0; r < n_ranges; ++r) rec[r] = RangeRec{0, range_xy[2 * r], range_xy[2 * r + 1], -1};
    const int64_t nact = n_ranges, off[2] = {0, n_ranges};
    if (n_ranges > 0 &&
        cudaMemcpyAsync(w.rec.p, rec.data(), sizeof(RangeRec) * n_ranges, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      rc = FIC_ECUDA;
    if (!rc && (cudaMemcpyAsync(w.n_act.p, &nact, sizeof(int64_t), cudaMemcpyHostToDevice, st) ||
                cudaMemcpyAsync(w.act_off.p, off, sizeof(off), cudaMemcpyHostToDevice, st) ||
                cudaMemcpyAsync(w.act_cnt.p, &nact, sizeof(int64_t), cudaMemcpyHostToDevice, st)))
      rc = FIC_ECUDA;
    if (!rc) rc = level_match(ctx, w, *params, 0, m->status.as<uint32_t>(), st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = FIC_ECUDA;  // host arrays above
  }
  // drop the borrowed buffers before any release
  w.pool.img = DevBuf(); w.pool.sel = DevBuf(); w.pool.slot_off = DevBuf();
  w.pool.bpack = DevBuf(); w.pool.b32 = DevBuf(); w.pool.dom = DevBuf(); w.pool.domf = DevBuf();
  w.pool.umax = DevBuf();
  w.pool.sd = DevBuf(); w.pool.sq = DevBuf(); w.pool.off = DevBuf();
  if (rc) {
    fic_matches_free(m);
    return rc;
  }
  *out = m;
  return FIC_OK;
}

int fic_matches_copy(const fic_matches* m, fic_match* host_out, size_t cap, size_t* count) {
  if (!m || (!host_out && cap > 0)) return FIC_EINVAL;
  int rc = sync_and_status(m->status, m->st);
  if (rc) return rc;
  if (count) *count = (size_t)m->n;
  if (cap < (size_t)m->n) return FIC_ERANGE;
  if (m->n > 0)
    FIC_CUDA_TRY(cudaMemcpy(host_out, m->ws.res.p, sizeof(fic_match) * m->n, cudaMemcpyDeviceToHost));
  return FIC_OK;
}

void fic_matches_free(fic_matches* m) {
  if (!m) return;
  cudaStreamSynchronize(m->st);
  m->ws.release_all();
  m->status.release();
  delete m;
}

// ------------------------------------------------------------ encoder
static int code_setup(fic_ctx* ctx, const fic_image* imgs, int n_images, const fic_params* params,
                      fic_code* c) {
  c->ctx = ctx;
  c->prm = *params;
  c->n_images = n_images;
  c->n_levels = params->single_level ? 1 : params->n_levels;
  c->ims.assign(imgs, imgs + n_images);
  c->dims = c->staging.device_view(c->ims);
  const size_t off_bytes = sizeof(int64_t) * 4 * (size_t)(n_images + 1);
  if (c->summary.reserve(off_bytes + 16)) return FIC_ENOMEM;
  c->status.p = (uint8_t*)c->summary.p + off_bytes;
  c->status.bytes = 16;
  for (int l = 0; l < c->n_levels; ++l) {
    const int B = params->range_size0 >> l;
    LevelWs& w = c->lv[l];
    pool_geometry(w.pool, c->dims, B, params->domain_step);
    w.pool.nsm = ctx->nsm;
    int rc = level_alloc(ctx, w, c->dims, B, ranges_at(c->dims, B), *params);
    if (!rc) rc = pool_alloc(w.pool);
    if (rc) return rc;
    w.code_off.release();  // the level's offsets live in the summary
    w.code_off.p = c->summary.as<int64_t>() + (size_t)l * (n_images + 1);
    w.code_off.bytes = sizeof(int64_t) * (size_t)(n_images + 1);
    // level 0's pool is on the critical path: the greatest priority; the
    // later levels' pools the least, so the level chain's kernels go first
    int lo = 0, hi = 0;
    FIC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    FIC_CUDA_TRY(cudaStreamCreateWithPriority(&c->side[l], cudaStreamNonBlocking, l == 0 ? hi : lo));
    FIC_CUDA_TRY(cudaEventCreateWithFlags(&c->pool_ev[l], cudaEventDisableTiming));
  }
  FIC_CUDA_TRY(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
  return FIC_OK;
}

static bool code_compatible(const fic_code* c, const fic_image* imgs, int n_images,
                            const fic_params* p) {
  if (c->n_images != n_images || memcmp(&c->prm, p, sizeof(fic_params)) != 0) return false;
  for (int i = 0; i < n_images; ++i)
    if (c->ims[i].width != imgs[i].width || c->ims[i].height != imgs[i].height ||
        c->ims[i].host != imgs[i].host)
      return false;
  return true;
}

int fic_encode(fic_ctx* ctx, const fic_image* imgs, int n_images, const fic_params* params,
               void* stream, fic_code** out) {
  if (!ctx || !imgs || !out || n_images < 1 || n_images > kMaxImages || !params)
    return FIC_EINVAL;
  if (const int pc = check_params(params)) return pc;
  *out = nullptr;
  for (int i = 0; i < n_images; ++i)
    if (!valid_image(imgs[i], params->range_size0)) return FIC_EINVAL;
  cudaSetDevice(ctx->device);
  fic_code* c = new (std::nothrow) fic_code();
  if (!c) return FIC_ENOMEM;
  int rc = code_setup(ctx, imgs, n_images, params, c);
  if (!rc) rc = encode_enqueue(c, (cudaStream_t)stream);
  if (rc) {
    fic_code_free(c);
    return rc;
  }
  *out = c;
  return FIC_OK;
}

int fic_encode_again(fic_ctx* ctx, const fic_image* imgs, int n_images, const fic_params* params,
                     void* stream, fic_code* code) {
  if (!ctx || !imgs || !code || code->ctx != ctx || !params) return FIC_EINVAL;
  if (const int pc = check_params(params)) return pc;
  if (!code_compatible(code, imgs, n_images, params)) return FIC_EINVAL;
  for (int i = 0; i < n_images; ++i)
    if (!valid_image(imgs[i], params->range_size0)) return FIC_EINVAL;
  cudaSetDevice(ctx->device);
  code->ims.assign(imgs, imgs + n_images);
  code->dims = code->staging.device_view(code->ims);
  for (auto& v : code->h_code_off) v.clear();
  if (stream) return encode_graph(code, (cudaStream_t)stream);
  return encode_enqueue(code, (cudaStream_t)stream);
}

int fic_code_set_profiling(fic_code* code, int on) {
  if (!code) return FIC_EINVAL;
  cudaSetDevice(code->ctx->device);
  if (on && !code->ev[0][0]) {
    for (auto& lv : code->ev)
      for (auto& e : lv) FIC_CUDA_TRY(cudaEventCreate(&e));
    for (auto& lv : code->pev)
      for (auto& e : lv) FIC_CUDA_TRY(cudaEventCreate(&e));
  }
  if ((on != 0) != code->profile && code->graph) {  // the graph holds the old choice
    cudaGraphExecDestroy(code->graph);
    code->graph = nullptr;
  }
  code->profile = on != 0;
  return FIC_OK;
}

int fic_code_profile(const fic_code* code, float* ms, int cap) {
  if (!code || !ms || cap < 2 * code->n_levels) return FIC_EINVAL;
  if (!code->profile) return FIC_EINVAL;
  FIC_CUDA_TRY(cudaStreamSynchronize(code->st));
  for (int l = 0; l < code->n_levels; ++l) {
    FIC_CUDA_TRY(cudaEventElapsedTime(&ms[2 * l], code->ev[l][1], code->ev[l][2]));
    FIC_CUDA_TRY(cudaEventElapsedTime(&ms[2 * l + 1], code->ev[l][0], code->ev[l][3]));
  }
  return FIC_OK;
}

int fic_code_pool_profile(const fic_code* code, float* ms, int cap) {
  if (!code || !ms || cap < code->n_levels) return FIC_EINVAL;
  if (!code->profile) return FIC_EINVAL;
  FIC_CUDA_TRY(cudaStreamSynchronize(code->st));
  for (int l = 0; l < code->n_levels; ++l)
    FIC_CUDA_TRY(cudaEventElapsedTime(&ms[l], code->pev[l][0], code->pev[l][1]));
  return FIC_OK;
}

int fic_code_schedule(const fic_code* code, int32_t* out, int cap) {
  if (!code || !out || cap < 2 * code->n_levels) return FIC_EINVAL;
  for (int l = 0; l < code->n_levels; ++l) {
    out[2 * l] = code->lv[l].items_per_cta;
    out[2 * l + 1] = code->lv[l].groups_per_tile;
  }
  return FIC_OK;
}

int fic_code_graph_kernels(const fic_code* code, int64_t* n) {
  if (!code || !n) return FIC_EINVAL;
  *n = code->graph ? code->graph_kernels : -1;
  return FIC_OK;
}

// The code offsets of every level and the status of the last encode, in one
// copy after the encode's stream has finished (cached until the next encode).
static int code_offsets(fic_code* c) {
  if (!c->h_code_off[0].empty()) return FIC_OK;
  FIC_CUDA_TRY(cudaStreamSynchronize(c->st));
  const size_t per = (size_t)c->n_images + 1;
  std::vector<int64_t> h(4 * per + 2);
  FIC_CUDA_TRY(cudaMemcpy(h.data(), c->summary.p, c->summary.bytes, cudaMemcpyDeviceToHost));
  uint32_t s = 0;
  memcpy(&s, &h[4 * per], sizeof(s));
  if (s & kStatusTimeout) return FIC_ETIMEOUT;
  if (s & kStatusOverflow) return FIC_ERANGE;
  for (int l = 0; l < c->n_levels; ++l)
    c->h_code_off[l].assign(h.begin() + l * per, h.begin() + (l + 1) * per);
  return FIC_OK;
}

int fic_code_count(const fic_code* code, int image_idx, size_t* count) {
  if (!code || !count || image_idx < 0 || image_idx >= code->n_images) return FIC_EINVAL;
  fic_code* c = const_cast<fic_code*>(code);
  cudaSetDevice(c->ctx->device);
  int rc = code_offsets(c);
  if (rc) return rc;
  size_t s = 0;
  for (int l = 0; l < c->n_levels; ++l)
    s += (size_t)(c->h_code_off[l][image_idx + 1] - c->h_code_off[l][image_idx]);
  *count = s;
  return FIC_OK;
}

int fic_code_get(const fic_code* code, int image_idx, fic_transform* host_out, size_t cap,
                 size_t* count) {
  size_t total = 0;
  int rc = fic_code_count(code, image_idx, &total);
  if (rc) return rc;
  if (count) *count = total;
  if (cap < total) return FIC_ERANGE;
  if (total && !host_out) return FIC_EINVAL;
  fic_code* c = const_cast<fic_code*>(code);
  // one asynchronous copy per level on the encode's stream, one wait (the
  // copies run as DMA straight into host_out when it is page-locked)
  size_t o = 0;
  for (int l = 0; l < c->n_levels; ++l) {
    const int64_t a = c->h_code_off[l][image_idx], b = c->h_code_off[l][image_idx + 1];
    if (b > a)
      FIC_CUDA_TRY(cudaMemcpyAsync(host_out + o, c->lv[l].codes.as<fic_transform>() + a,
                                   sizeof(fic_transform) * (size_t)(b - a),
                                   cudaMemcpyDeviceToHost, c->st));
    o += (size_t)(b - a);
  }
  FIC_CUDA_TRY(cudaStreamSynchronize(c->st));
  return FIC_OK;
}

int fic_code_stats(const fic_code* code, int image_idx, fic_level_stats* host_out, int cap) {
  if (!code || !host_out || image_idx < 0 || image_idx >= code->n_images) return FIC_EINVAL;
  if (cap < code->n_levels) return FIC_ERANGE;
  fic_code* c = const_cast<fic_code*>(code);
  cudaSetDevice(c->ctx->device);
  FIC_CUDA_TRY(cudaDeviceSynchronize());
  int rc = sync_and_status(c->status, nullptr);
  if (rc) return rc;
  for (int l = 0; l < c->n_levels; ++l) {
    const LevelWs& w = c->lv[l];
    SelState s{};
    int64_t ac = 0;
    int32_t acc = 0;
    FIC_CUDA_TRY(cudaMemcpy(&s, w.pool.sel.as<SelState>() + image_idx, sizeof(s),
                            cudaMemcpyDeviceToHost));
    FIC_CUDA_TRY(cudaMemcpy(&ac, w.act_cnt.as<int64_t>() + image_idx, sizeof(ac),
                            cudaMemcpyDeviceToHost));
    FIC_CUDA_TRY(cudaMemcpy(&acc, w.acc_cnt.as<int32_t>() + image_idx, sizeof(acc),
                            cudaMemcpyDeviceToHost));
    fic_level_stats& o = host_out[l];
    o.size = w.B;
    o.pool_size = (int32_t)(w.pool.h_off[image_idx + 1] - w.pool.h_off[image_idx]);
    o.n_kept = s.nkept;
    o.fallback = s.fallback;
    o.thr_key = s.thr;
    o.n_active = (int32_t)ac;
    o.n_accepted = acc;
    o.matches = (double)ac * (double)s.nkept * 8.0;
  }
  return FIC_OK;
}

int fic_code_quantize_o(fic_code* code, int o_bits) {
  if (!code || o_bits < 1 || o_bits > 16) return FIC_EINVAL;
  cudaSetDevice(code->ctx->device);
  for (int l = 0; l < code->n_levels; ++l) {
    LevelWs& w = code->lv[l];
    // the level's saved maps: code_off[n_images] of them
    int rc = launch_quantize_o(w.codes.as<fic_transform>(),
                               w.code_off.as<int64_t>() + code->n_images, w.cap, o_bits, code->st);
    if (rc) return rc;
  }
  return FIC_OK;
}

int fic_code_bits(const fic_code* code, int image_idx, int o_bits, int64_t* bits) {
  if (!code || !bits || o_bits < 1 || o_bits > 16) return FIC_EINVAL;
  if (code->prm.s_mode == FIC_S_EXACT) return FIC_EINVAL;  // s from no finite set
  fic_level_stats st[4];
  int rc = fic_code_stats(code, image_idx, st, 4);
  if (rc) return rc;
  auto ceil_log2 = [](int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
  };
  int64_t total = 0;
  for (int l = 0; l < code->n_levels; ++l) {
    SSet S;
    make_sset(code->prm.s_mode, code->prm.grid_samples, st[l].size, &S);
    if (l < code->n_levels - 1) total += st[l].n_active;  // kept or split
    total += (int64_t)st[l].n_accepted * (ceil_log2(st[l].pool_size) + 3 + ceil_log2(S.m) + o_bits);
  }
  *bits = total;
  return FIC_OK;
}

void fic_code_free(fic_code* c) {
  if (!c) return;
  if (c->ctx) cudaSetDevice(c->ctx->device);
  cudaDeviceSynchronize();
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto& lv : c->ev)
    for (auto& e : lv)
      if (e) cudaEventDestroy(e);
  for (auto& lv : c->pev)
    for (auto& e : lv)
      if (e) cudaEventDestroy(e);
  for (int l = 0; l < 4; ++l) {
    if (c->pool_ev[l]) cudaEventDestroy(c->pool_ev[l]);
    if (c->side[l]) cudaStreamDestroy(c->side[l]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  for (auto& w : c->lv) {  // a level's offsets alias the summary once set up
    const uint8_t* q = (const uint8_t*)w.code_off.p;
    const uint8_t* b = (const uint8_t*)c->summary.p;
    if (q && b && q >= b && q < b + c->summary.bytes) w.code_off = DevBuf();
  }
  for (auto& w : c->lv) w.release_all();
  c->rng_off.release();
  c->staging.buf.release();
  c->dec.release();
  c->status = DevBuf();  // alias of the summary
  c->summary.release();
  delete c;
}

int fic_decode(fic_ctx* ctx, const fic_code* code, int image_idx, int max_iters, double tol,
               uint8_t* out, int out_pitch, int out_host, void* stream, int* iters_done) {
  if (!ctx || !code || !out || image_idx < 0 || image_idx >= code->n_images || max_iters < 0)
    return FIC_EINVAL;
  fic_code* c = const_cast<fic_code*>(code);
  const int W = c->ims[image_idx].width, H = c->ims[image_idx].height;
  if (out_pitch < W) return FIC_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = code_offsets(c);
  if (rc) return rc;
  // gather this image's codes of every level into one array
  size_t total = 0;
  for (int l = 0; l < c->n_levels; ++l)
    total += (size_t)(c->h_code_off[l][image_idx + 1] - c->h_code_off[l][image_idx]);
  DevBuf gathered;
  if (gathered.reserve(sizeof(fic_transform) * (total ? total : 1))) return FIC_ENOMEM;
  size_t o = 0;
  for (int l = 0; l < c->n_levels; ++l) {
    const int64_t a = c->h_code_off[l][image_idx], b = c->h_code_off[l][image_idx + 1];
    if (b > a)
      cudaMemcpyAsync(gathered.as<fic_transform>() + o, c->lv[l].codes.as<fic_transform>() + a,
                      sizeof(fic_transform) * (size_t)(b - a), cudaMemcpyDeviceToDevice, st);
    o += (size_t)(b - a);
  }
  DevBuf dout;
  uint8_t* dptr = out;
  int dpitch = out_pitch;
  if (out_host) {
    if (dout.reserve((size_t)W * H)) {
      gathered.release();
      return FIC_ENOMEM;
    }
    dptr = dout.as<uint8_t>();
    dpitch = W;
  }
  rc = decode_run(gathered.as<fic_transform>(), (int64_t)total, W, H, max_iters, tol, c->dec, dptr,
                  dpitch, st);
  if (!rc && out_host &&
      cudaMemcpy2DAsync(out, out_pitch, dptr, W, W, H, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = FIC_ECUDA;
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = FIC_ECUDA;
  if (!rc) {
    int32_t ctl[4];  // done, iterations, a barrier wait that ran out
    if (cudaMemcpy(ctl, c->dec.ctl.p, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = FIC_ECUDA;
    else if (ctl[2])
      rc = FIC_ETIMEOUT;
    else if (iters_done)
      *iters_done = ctl[1];
  }
  gathered.release();
  dout.release();
  return rc;
}

}  // extern "C"
