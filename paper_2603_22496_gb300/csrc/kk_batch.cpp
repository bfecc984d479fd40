// kk_batch.cpp -- batched form: many frames of uneven size in one CUDA graph
// whose image formation is a single persistent launch.
//
// A batch is built from per-frame KK plans and the frames' device buffers.
// Its CUDA graph forks every frame's decomposition (spectrum, contraction,
// inverse; independent frames run concurrently on several capture streams),
// joins, resets a work counter and runs one persistent gather over the
// (frame, tile) work items of all frames, largest frames first.  The launch
// shape of that gather (tile rows, pairs per stage) is picked by timing the
// feasible shapes on the batch itself (the autotuner) or set by the caller.
// Volumetric frames form a second work list (tiles over every y slice) with
// its own persistent launch, counter and launch shape, after the first.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "kk_internal.h"

namespace {

constexpr int kCaptureStreams = 128;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

}  // namespace

// One persistent launch's work: the (frame, tile) items of the linear-array
// frames (vol = false) or of the volumetric ones, and its launch shape.
struct BatchList {
  bool vol = false;
  int2 *d_items = nullptr;
  int *d_counter = nullptr;
  size_t cap = 0;
  int n_frames = 0, n_items = 0, max_win = 0, rows = 4, stage = 16;
  float tuned_ms[16] = {};
  int tuned_cfg[16] = {};
  int n_tuned = 0;
};

struct kk_batch {
  int device = 0;
  std::vector<kk_batch_frame> frames;
  // device block: GatherArgs[n] | GatherVolArgs[n] | per list: int2 items[], int counter
  void *dev = nullptr;
  kk::GatherArgs *d_args = nullptr;
  kk::GatherVolArgs *d_vols = nullptr;
  std::vector<kk::GatherArgs> h_args;   // host copies, both lists' frames
  std::vector<kk::GatherVolArgs> h_vols;
  BatchList lists[2];                   // linear-array frames, volumetric frames
  int grid = 0;
  double pixel_pairs = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t graph_nodes = 0;
  cudaStream_t main_stream = nullptr;  // private: capture and autotuning
  cudaStream_t streams[kCaptureStreams] = {};
  cudaEvent_t fork = nullptr, join[kCaptureStreams] = {};
};

namespace kk {
namespace {

// window length and tile rows of one frame for a launch shape
int frame_window(const kk_plan &p, int rows) {
  const int tz = 4 * rows;
  double span = 0;
  for (size_t q = 0; q < p.h_bfA.size(); ++q)
    span = std::max(span, std::fabs(p.h_bfA[q]) * (kTileX - 1) + p.h_bfB[q] * (tz - 1));
  return (int)std::ceil(span) + 4;
}

// Frame descriptors (into the host copies) and work items of a launch shape
// for one list; false if a frame's window does not fit the shape.
bool build_items(kk_batch &b, BatchList &L, int rows, int stage, std::vector<int2> &items, int &max_win) {
  items.clear();
  max_win = 0;
  std::vector<std::pair<double, int>> order;
  for (size_t f = 0; f < b.frames.size(); ++f) {
    const kk_plan &p = *b.frames[f].plan;
    if (p.vol != L.vol) continue;
    const int win = frame_window(p, rows);
    if (!gather_config_supported(rows, stage, win)) return false;
    max_win = std::max(max_win, win);
    GatherArgs a = gather_args(p, (const float2 *)b.frames[f].d_rf_theta, (float2 *)b.frames[f].d_B,
                               b.frames[f].d_I);
    a.win = win;
    a.split = 1;
    a.tiles_x = (p.grid.nx + kTileX - 1) / kTileX;
    b.h_args[f] = a;
    if (L.vol) {
      GatherVolArgs v = gather_vol_args(p);
      v.tiles_xz = a.tiles_x * ((p.grid.nz + 4 * rows - 1) / (4 * rows));
      b.h_vols[f] = v;
    }
    order.push_back({(double)p.P, (int)f});
  }
  if (!gather_config_supported(rows, stage, max_win)) return false;
  // largest frames (most pairs per tile) first
  std::stable_sort(order.begin(), order.end(), [](auto &x, auto &y) { return x.first > y.first; });
  for (auto &o : order) {
    const kk_plan &p = *b.frames[o.second].plan;
    const int tiles = b.h_args[o.second].tiles_x * ((p.grid.nz + 4 * rows - 1) / (4 * rows)) * (L.vol ? p.ny : 1);
    for (int t = 0; t < tiles; ++t) items.push_back(make_int2(o.second, t));
  }
  return true;
}

kk_status upload_items(kk_batch &b, BatchList &L, const std::vector<int2> &items, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b.d_args, b.h_args.data(), sizeof(GatherArgs) * b.h_args.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.d_vols, b.h_vols.data(), sizeof(GatherVolArgs) * b.h_vols.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(L.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "batch descriptor upload");
}

kk_status enqueue_gather(kk_batch &b, const BatchList &L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(L.d_counter, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_kk_gather_batch(L.rows, L.stage, b.d_args, L.vol ? b.d_vols : nullptr, L.d_items, L.n_items,
                               L.d_counter, L.max_win, b.grid, s);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "batched gather launch");
}

kk_status select_shape(kk_batch &b, BatchList &L, int rows, int stage, cudaStream_t s) {
  std::vector<int2> items;
  int max_win = 0;
  if (!build_items(b, L, rows, stage, items, max_win)) {
    set_error(std::string("launch shape does not fit the batch's ") + (L.vol ? "volumetric " : "") + "windows");
    return KK_ERR_UNSUPPORTED;
  }
  if (items.size() > L.cap) {
    set_error("work list larger than allocated");
    return KK_ERR_INVALID_ARG;
  }
  L.rows = rows;
  L.stage = stage;
  L.max_win = max_win;
  L.n_items = (int)items.size();
  return upload_items(b, L, items, s);
}

kk_status capture_graph(kk_batch &b, cudaStream_t s) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b.exec = nullptr;
  b.graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  kk_status st = KK_OK;
  e = cudaEventRecord(b.fork, s);
  for (int k = 0; k < kCaptureStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b.streams[k], b.fork, 0);
  for (size_t f = 0; f < b.frames.size() && e == cudaSuccess && st == KK_OK; ++f) {
    const kk_batch_frame &fr = b.frames[f];
    st = enqueue_decompose(fr.plan, fr.d_rf, fr.d_rf_theta, fr.d_workspace, b.streams[f % kCaptureStreams],
                           true);
  }
  for (int k = 0; k < kCaptureStreams && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b.join[k], b.streams[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.join[k], 0);
  }
  for (const BatchList &L : b.lists)
    if (e == cudaSuccess && st == KK_OK && L.n_items > 0) st = enqueue_gather(b, L, s);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (st != KK_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e != cudaSuccess ? e : e2, "graph capture");
  }
  e = cudaGraphInstantiate(&b.exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "graph instantiate");
  }
  b.graph = g;
  cudaGraphGetNodes(g, nullptr, &b.graph_nodes);
  return KK_OK;
}

// Time one list's batched gather alone for every feasible shape; keep the
// fastest.
kk_status autotune(kk_batch &b, BatchList &L, cudaStream_t s) {
  static const int cands[][2] = {{4, 16}, {4, 8}, {8, 8}, {8, 4}, {2, 16}, {4, 4}, {2, 8}};
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  int best_i = -1;
  L.n_tuned = 0;
  for (int c = 0; c < (int)(sizeof(cands) / sizeof(cands[0])); ++c) {
    if (select_shape(b, L, cands[c][0], cands[c][1], s) != KK_OK) continue;
    float ms = 0;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {  // first launch warms up
      cudaEventRecord(t0, s);
      ok = enqueue_gather(b, L, s) == KK_OK;
      cudaEventRecord(t1, s);
      if (cudaEventSynchronize(t1) != cudaSuccess) ok = false;
      float m = 0;
      cudaEventElapsedTime(&m, t0, t1);
      if (rep > 0) ms += m;
    }
    if (!ok) continue;
    ms /= 2;
    L.tuned_ms[L.n_tuned] = ms;
    L.tuned_cfg[L.n_tuned] = cands[c][0] * 100 + cands[c][1];
    ++L.n_tuned;
    if (ms < best) {
      best = ms;
      best_i = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaGetLastError();
  if (best_i < 0) {
    set_error(std::string("no launch shape fits this batch's ") + (L.vol ? "volumetric " : "") + "frames");
    return KK_ERR_UNSUPPORTED;
  }
  return select_shape(b, L, cands[best_i][0], cands[best_i][1], s);
}

void destroy(kk_batch *b) {
  if (!b) return;
  DeviceGuard guard(b->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int k = 0; k < kCaptureStreams; ++k) {
    if (b->streams[k]) cudaStreamDestroy(b->streams[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->main_stream) cudaStreamDestroy(b->main_stream);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

}  // namespace
}  // namespace kk

using namespace kk;

extern "C" {

kk_status kk_batch_create(kk_batch **out, const kk_batch_frame *frames, int32_t n_frames,
                          int32_t shape, void *stream) {
  if (!out || !frames || n_frames < 1) { set_error("null argument or n_frames < 1"); return KK_ERR_INVALID_ARG; }
  *out = nullptr;
  const int device = frames[0].plan ? frames[0].plan->device : -1;
  for (int f = 0; f < n_frames; ++f) {
    const kk_batch_frame &fr = frames[f];
    if (!fr.plan || fr.plan->is_das) { set_error("every frame needs a KK plan"); return KK_ERR_INVALID_ARG; }
    if (fr.plan->device != device) { set_error("all plans must live on one device"); return KK_ERR_INVALID_ARG; }
    if (!fr.d_rf || !fr.d_rf_theta || !fr.d_B || !fr.d_workspace) { set_error("null frame buffer"); return KK_ERR_INVALID_ARG; }
    if (fr.plan->compound != KK_COMPOUND_NONE && !fr.d_I) { set_error("compound mode set but I is null"); return KK_ERR_INVALID_ARG; }
    if ((uintptr_t)fr.d_rf % 16 || (uintptr_t)fr.d_rf_theta % 16 || (uintptr_t)fr.d_workspace % kAlign) {
      set_error("frame buffers must be 16-byte aligned (workspace 256)");
      return KK_ERR_INVALID_ARG;
    }
  }
  if (shape != 0 && !((shape / 100 == 2 || shape / 100 == 4 || shape / 100 == 8) &&
                      (shape % 100 == 4 || shape % 100 == 8 || shape % 100 == 16))) {
    set_error("shape must be 0 (autotune) or rows*100+stage with rows in {2,4,8}, stage in {4,8,16}");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(device);
  kk_batch *b = new (std::nothrow) kk_batch();
  if (!b) { set_error("host allocation failed"); return KK_ERR_OOM; }
  b->device = device;
  b->frames.assign(frames, frames + n_frames);
  b->h_args.assign(n_frames, GatherArgs{});
  b->h_vols.assign(n_frames, GatherVolArgs{});
  b->lists[1].vol = true;
  cudaStream_t s = (cudaStream_t)stream;
  // work list capacities: the most tiles any shape produces (rows = 2)
  for (int f = 0; f < n_frames; ++f) {
    const kk_plan &p = *frames[f].plan;
    BatchList &L = b->lists[p.vol ? 1 : 0];
    L.cap += (size_t)((p.grid.nx + kTileX - 1) / kTileX) * ((p.grid.nz + 7) / 8) * p.ny;
    ++L.n_frames;
    b->pixel_pairs += (double)p.P * p.grid.nx * p.grid.nz * p.ny;
  }
  const size_t o_vols = align_up(sizeof(GatherArgs) * n_frames);
  const size_t o_list0 = o_vols + align_up(sizeof(GatherVolArgs) * n_frames);
  const size_t o_list1 = o_list0 + align_up(sizeof(int2) * b->lists[0].cap) + kAlign;
  const size_t bytes = o_list1 + align_up(sizeof(int2) * b->lists[1].cap) + kAlign;
  cudaError_t e = cudaMalloc(&b->dev, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    set_error("batch descriptor allocation failed");
    return KK_ERR_OOM;
  }
  unsigned char *base = (unsigned char *)b->dev;
  b->d_args = (GatherArgs *)base;
  b->d_vols = (GatherVolArgs *)(base + o_vols);
  b->lists[0].d_items = (int2 *)(base + o_list0);
  b->lists[0].d_counter = (int *)(base + o_list0 + align_up(sizeof(int2) * b->lists[0].cap));
  b->lists[1].d_items = (int2 *)(base + o_list1);
  b->lists[1].d_counter = (int *)(base + o_list1 + align_up(sizeof(int2) * b->lists[1].cap));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  b->grid = 8 * sms;  // persistent: up to 8 resident CTAs per SM
  for (int k = 0; k < kCaptureStreams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->main_stream, cudaStreamNonBlocking);
  // work already queued on the caller's stream (e.g. filling the buffers)
  // completes before the autotuner runs
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    kk_status st = cuda_fail(e, "batch stream setup");
    destroy(b);
    return st;
  }
  cudaStream_t ms = b->main_stream;
  kk_status st = KK_OK;
  for (BatchList &L : b->lists)
    if (st == KK_OK && L.n_frames > 0)
      st = (shape == 0) ? autotune(*b, L, ms) : select_shape(*b, L, shape / 100, shape % 100, ms);
  if (st == KK_OK) st = capture_graph(*b, ms);
  if (st == KK_OK) {
    e = cudaStreamSynchronize(ms);
    if (e != cudaSuccess) st = cuda_fail(e, "batch setup");
  }
  if (st != KK_OK) {
    destroy(b);
    return st;
  }
  *out = b;
  return KK_OK;
}

kk_status kk_batch_run(kk_batch *b, void *stream) {
  NvtxRange range("kk_batch_run");
  if (!b || !b->exec) { set_error("null batch"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(b->device);
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "graph launch");
}

kk_status kk_batch_get_info(const kk_batch *b, kk_batch_info *info) {
  if (!b || !info) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  std::memset(info, 0, sizeof(*info));
  const BatchList &L = b->lists[0], &V = b->lists[1];
  info->n_frames = (int32_t)b->frames.size();
  info->n_items = L.n_items;
  info->rows = L.n_frames ? L.rows : 0;
  info->stage = L.n_frames ? L.stage : 0;
  info->max_window = L.max_win;
  info->grid = b->grid;
  info->graph_nodes = (int32_t)b->graph_nodes;
  info->pixel_pairs = b->pixel_pairs;
  info->n_tuned = L.n_tuned;
  for (int i = 0; i < L.n_tuned && i < 16; ++i) {
    info->tuned_shape[i] = L.tuned_cfg[i];
    info->tuned_ms[i] = L.tuned_ms[i];
  }
  info->n_volume_frames = V.n_frames;
  info->n_items_volume = V.n_items;
  info->rows_volume = V.n_frames ? V.rows : 0;
  info->stage_volume = V.n_frames ? V.stage : 0;
  info->max_window_volume = V.max_win;
  return KK_OK;
}

void kk_batch_destroy(kk_batch *b) { destroy(b); }

}  // extern "C"
