// kk_stream.cpp -- streaming decomposition (include/kkstream.h).
//
// The far-field decomposition of Eq. (compression) is independent per
// transmit: the spectrum of transmit i's channels, the per-bin contraction
// of those channels against the receive angles, and the inverse transforms
// of the pairs (i, o) touch no other transmit's data.  So a frame can be
// decomposed group by group as its transmit events arrive, with the same
// kernels as kk_decompose run on a plan copy whose transmit count is the
// group's, and the image formation of Eq. (KK) can run for the previous
// frame meanwhile.
//
// Device memory (one allocation):
//   ring    [R][G][L][T] samples   R groups of events (copies run up to R - 1
//                                  groups ahead of the decomposition)
//   X, Y    one group's spectrum [F][G][L] and contraction output [F][G][Mu]
//   rt      [2][P][T] cfloat       rf_theta of two frames in flight
//   ws      [2] plan workspaces    image formation of two frames in flight
//   tables  slot rows 0..G-1; per group: Y column, rf_theta row and weight
//           of each of its pairs
// Dependencies are CUDA events between three streams (copy, decomposition,
// image); nothing spins on the device.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "kk_internal.h"
#include "kkstream.h"

using namespace kk;

namespace {

constexpr size_t kAlignS = 256;
size_t up(size_t v) { return (v + kAlignS - 1) / kAlignS * kAlignS; }

struct Group {
  kk_plan sub;             // plan copy with Nu = this group's transmits
  int first_tu = 0, n_tx = 0, n_pairs = 0;
  int32_t *d_col = nullptr;    // Y column of each pair: (tu - first_tu) * Mu + ou
  bool col_identity = false;   // d_col[j] == j
  int32_t *d_orow = nullptr;   // rf_theta row (caller's pair order)
  float *d_w = nullptr;        // pair weight (null without weights)
};

}  // namespace

struct kk_stream {
  const kk_plan *plan = nullptr;
  int device = 0;
  int G = 1, n_groups = 0;
  size_t ev_bytes = 0;
  std::vector<Group> groups;
  std::vector<int> tu_of_row;     // transmit position of each rf row, -1 unused
  unsigned char *block = nullptr;
  size_t block_bytes = 0;
  int R = 2;                              // ring depth in groups
  std::vector<unsigned char *> ring;
  void *X = nullptr;
  float2 *Y = nullptr;
  float2 *rt[2] = {nullptr, nullptr};
  void *ws[2] = {nullptr, nullptr};
  int32_t *d_slot_rows = nullptr;
  cudaStream_t s_copy = nullptr, s_dec = nullptr, s_img = nullptr;
  std::vector<cudaEvent_t> ev_copied, ev_dec;   // per ring group
  std::vector<char> dec_pending;
  cudaEvent_t ev_frame_dec[2] = {}, ev_img[2] = {};
  cudaEvent_t ev_ext = nullptr;  // caller-stream work the image stream waits for
  bool img_pending[2] = {false, false};
  // state of the frame being pushed
  long long frame = 0;       // frames ended so far
  int next_row = 0;          // lowest row the next push may carry
  int next_tu = 0;           // transmits in use pushed so far in this frame
  long long group_seq = 0;   // groups started (ring group = group_seq % R)
  // copy run not yet issued: consecutive events contiguous in both the
  // source and the ring go out as one copy when the group fills (or the run
  // breaks)
  const unsigned char *run_src = nullptr;
  unsigned char *run_dst = nullptr;
  size_t run_bytes = 0;
  cudaMemcpyKind run_kind = cudaMemcpyHostToDevice;
  // statistics
  long long events = 0, dropped = 0, groups_run = 0, copies = 0;

  ~kk_stream() {
    if (s_copy) cudaStreamSynchronize(s_copy);
    if (s_dec) cudaStreamSynchronize(s_dec);
    if (s_img) cudaStreamSynchronize(s_img);
    for (cudaEvent_t e : ev_copied)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_dec)
      if (e) cudaEventDestroy(e);
    for (int b = 0; b < 2; ++b) {
      if (ev_frame_dec[b]) cudaEventDestroy(ev_frame_dec[b]);
      if (ev_img[b]) cudaEventDestroy(ev_img[b]);
    }
    if (ev_ext) cudaEventDestroy(ev_ext);
    if (s_copy) cudaStreamDestroy(s_copy);
    if (s_dec) cudaStreamDestroy(s_dec);
    if (s_img) cudaStreamDestroy(s_img);
    if (block) cudaFree(block);
  }
};

namespace {

int sample_bytes(const kk_plan &p) { return p.rf_dtype == KK_RF_I16 ? 2 : 4; }

size_t spectrum_bytes_of(const kk_plan &p, int n_tx) {
  return (size_t)p.F * n_tx * p.L * spectrum_bytes(p.precision);
}

cudaError_t flush_copy(kk_stream *s) {
  if (!s->run_bytes) return cudaSuccess;
  const cudaError_t e = cudaMemcpyAsync(s->run_dst, s->run_src, s->run_bytes, s->run_kind, s->s_copy);
  s->run_bytes = 0;
  ++s->copies;
  return e;
}

// `extend`: src continues the caller's block of the previous event (only a
// block handed over by kk_stream_push_many is known to be one allocation;
// separately pushed buffers may be adjacent yet belong to different ones)
cudaError_t add_copy(kk_stream *s, unsigned char *dst, const void *src, cudaMemcpyKind kind, bool extend) {
  const unsigned char *sp = static_cast<const unsigned char *>(src);
  if (extend && s->run_bytes && kind == s->run_kind && sp == s->run_src + s->run_bytes &&
      dst == s->run_dst + s->run_bytes) {
    s->run_bytes += s->ev_bytes;
    return cudaSuccess;
  }
  const cudaError_t e = flush_copy(s);
  s->run_src = sp;
  s->run_dst = dst;
  s->run_bytes = s->ev_bytes;
  s->run_kind = kind;
  return e;
}

// Enqueues the decomposition of group g (just completed) on s_dec.
kk_status run_group(kk_stream *s, int g) {
  NvtxRange range("kk_stream/decompose_group");
  const int b = (int)(s->group_seq % s->R);
  Group &gr = s->groups[g];
  cudaError_t e = flush_copy(s);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream: copy");
  e = cudaEventRecord(s->ev_copied[b], s->s_copy);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_dec, s->ev_copied[b], 0);
  if (e == cudaSuccess && g == 0 && s->img_pending[s->frame % 2])
    e = cudaStreamWaitEvent(s->s_dec, s->ev_img[s->frame % 2], 0);  // rf_theta buffer free again
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream: event");
  e = launch_spectrum(gr.sub, s->ring[b], s->X, gr.n_tx, s->d_slot_rows, s->s_dec);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream: spectrum launch");
  e = launch_shear(gr.sub, s->X, s->Y, s->s_dec);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream: shear launch");
  e = launch_inverse(gr.sub, s->Y, gr.n_tx * gr.sub.Mu, gr.col_identity ? nullptr : gr.d_col, gr.n_pairs,
                     s->rt[s->frame % 2], s->s_dec,
                     gr.d_w, gr.d_orow);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream: inverse launch");
  e = cudaEventRecord(s->ev_dec[b], s->s_dec);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream: event");
  s->dec_pending[b] = true;
  ++s->group_seq;
  ++s->groups_run;
  return KK_OK;
}

kk_status push_event(kk_stream *s, int32_t tx_row, const void *h_event, const void *d_event, bool extend);

}  // namespace

extern "C" {

kk_status kk_stream_create(kk_stream **out, const kk_plan *plan, int32_t group, int32_t ring_groups) {
  if (!out || !plan) {
    set_error("kk_stream_create: null argument");
    return KK_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (plan->is_das) {
    set_error("kk_stream_create: expected a KK plan");
    return KK_ERR_INVALID_ARG;
  }
  if (group < 1 || group > plan->Nu) {
    set_error("kk_stream_create: group must be in [1, transmits in use = " + std::to_string(plan->Nu) + "]");
    return KK_ERR_INVALID_ARG;
  }
  if (ring_groups < 2 || ring_groups > 64) {
    set_error("kk_stream_create: ring_groups must be in [2, 64]");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  if (!guard.ok) {
    set_error("kk_stream_create: cannot select the plan's device");
    return KK_ERR_CUDA;
  }
  kk_stream *s = new (std::nothrow) kk_stream;
  if (!s) {
    set_error("kk_stream_create: host allocation failed");
    return KK_ERR_OOM;
  }
  const kk_plan &p = *plan;
  s->plan = plan;
  s->device = plan->device;
  s->G = group;
  s->R = ring_groups;
  s->ring.assign(ring_groups, nullptr);
  s->ev_copied.assign(ring_groups, nullptr);
  s->ev_dec.assign(ring_groups, nullptr);
  s->dec_pending.assign(ring_groups, 0);
  s->n_groups = (p.Nu + group - 1) / group;
  s->ev_bytes = (size_t)p.L * p.T * sample_bytes(p);
  s->tu_of_row.assign(p.N, -1);
  for (int a = 0; a < p.Nu; ++a) s->tu_of_row[p.h_tx_used[a]] = a;

  // pairs of each group (caller's order kept within a group)
  std::vector<std::vector<int32_t>> col(s->n_groups), orow(s->n_groups);
  std::vector<std::vector<float>> w(s->n_groups);
  for (int q = 0; q < p.P; ++q) {
    const int tu = p.h_pair_tu[q], g = tu / group;
    col[g].push_back((tu - g * group) * p.Mu + p.h_pair_ou[q]);
    orow[g].push_back(q);
    if (!p.h_pair_w.empty()) w[g].push_back(p.h_pair_w[q]);
  }

  // one device block
  size_t off = 0;
  const size_t o_ring = off; off += (size_t)ring_groups * up((size_t)group * s->ev_bytes);
  const size_t o_X = off; off += up(spectrum_bytes_of(p, group));
  const size_t o_Y = off; off += up((size_t)p.F * group * p.Mu * sizeof(float2));
  const size_t o_rt = off; off += 2 * up((size_t)p.P * p.T * sizeof(float2));
  const size_t o_ws = off; off += 2 * up(p.ws_total);
  const size_t o_rows = off; off += up((size_t)group * sizeof(int32_t));
  std::vector<size_t> o_tab(s->n_groups);
  for (int g = 0; g < s->n_groups; ++g) {
    o_tab[g] = off;
    off += up(col[g].size() * sizeof(int32_t)) * 2 + up(w[g].size() * sizeof(float));
  }
  s->block_bytes = off;
  cudaError_t e = cudaMalloc(&s->block, off);
  if (e != cudaSuccess) {
    delete s;
    set_error("kk_stream_create: cannot allocate " + std::to_string(off) + " device bytes");
    return KK_ERR_OOM;
  }
  const size_t ring_stride = up((size_t)group * s->ev_bytes);
  for (int b = 0; b < ring_groups; ++b) s->ring[b] = s->block + o_ring + (size_t)b * ring_stride;
  s->X = s->block + o_X;
  s->Y = reinterpret_cast<float2 *>(s->block + o_Y);
  const size_t rt_stride = up((size_t)p.P * p.T * sizeof(float2));
  s->rt[0] = reinterpret_cast<float2 *>(s->block + o_rt);
  s->rt[1] = reinterpret_cast<float2 *>(s->block + o_rt + rt_stride);
  s->ws[0] = s->block + o_ws;
  s->ws[1] = s->block + o_ws + up(p.ws_total);
  s->d_slot_rows = reinterpret_cast<int32_t *>(s->block + o_rows);

  auto fail = [&](cudaError_t err, const char *what) {
    const kk_status st = cuda_fail(err, what);
    delete s;
    return st;
  };
  std::vector<int32_t> rows(group);
  for (int j = 0; j < group; ++j) rows[j] = j;
  e = cudaMemcpy(s->d_slot_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "kk_stream_create: table upload");
  s->groups.resize(s->n_groups);
  for (int g = 0; g < s->n_groups; ++g) {
    Group &gr = s->groups[g];
    gr.first_tu = g * group;
    gr.n_tx = std::min(group, p.Nu - gr.first_tu);
    gr.n_pairs = (int)col[g].size();
    gr.sub = p;
    gr.sub.Nu = gr.n_tx;
    unsigned char *base = s->block + o_tab[g];
    const size_t nb = up(col[g].size() * sizeof(int32_t));
    gr.d_col = reinterpret_cast<int32_t *>(base);
    gr.col_identity = true;  // the group's pair j reads column j of its Y (TMA-fed inverse)
    for (size_t j = 0; j < col[g].size() && gr.col_identity; ++j) gr.col_identity = col[g][j] == (int32_t)j;
    gr.d_orow = reinterpret_cast<int32_t *>(base + nb);
    gr.d_w = w[g].empty() ? nullptr : reinterpret_cast<float *>(base + 2 * nb);
    if (gr.n_pairs) {
      e = cudaMemcpy(gr.d_col, col[g].data(), col[g].size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(gr.d_orow, orow[g].data(), orow[g].size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && gr.d_w)
        e = cudaMemcpy(gr.d_w, w[g].data(), w[g].size() * sizeof(float), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return fail(e, "kk_stream_create: table upload");
    }
  }
  int lo = 0, hi = 0;
  e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->s_copy, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->s_dec, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->s_img, cudaStreamNonBlocking, lo);
  for (int b = 0; b < ring_groups && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&s->ev_copied[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_dec[b], cudaEventDisableTiming);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&s->ev_frame_dec[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_img[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_ext, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail(e, "kk_stream_create: streams and events");
  *out = s;
  return KK_OK;
}

kk_status kk_stream_push(kk_stream *s, int32_t tx_row, const void *h_event, const void *d_event) {
  return push_event(s, tx_row, h_event, d_event, false);
}

}  // extern "C"

namespace {

kk_status push_event(kk_stream *s, int32_t tx_row, const void *h_event, const void *d_event, bool extend) {
  if (!s) {
    set_error("kk_stream_push: null stream");
    return KK_ERR_INVALID_ARG;
  }
  const kk_plan &p = *s->plan;
  if (tx_row < s->next_row || tx_row >= p.N) {
    set_error("kk_stream_push: rows of a frame must increase within [0, n_tx) (got " + std::to_string(tx_row) +
              ", next allowed " + std::to_string(s->next_row) + ")");
    return KK_ERR_INVALID_ARG;
  }
  const int tu = s->tu_of_row[tx_row];
  if (tu >= 0 && s->next_tu == p.Nu) {
    set_error("kk_stream_push: the frame is complete; call kk_stream_end_frame first");
    return KK_ERR_INVALID_ARG;
  }
  if (tu >= 0 && tu != s->next_tu) {
    set_error("kk_stream_push: transmit row " + std::to_string(p.h_tx_used[s->next_tu]) +
              " is in use and was skipped");
    return KK_ERR_INVALID_ARG;
  }
  if (tu < 0) {  // a transmit the plan does not use: nothing to copy
    if (s->next_tu < p.Nu) {
      const int want = p.h_tx_used[s->next_tu];
      if (tx_row > want) {
        set_error("kk_stream_push: transmit row " + std::to_string(want) + " is in use and was skipped");
        return KK_ERR_INVALID_ARG;
      }
    }
    s->next_row = tx_row + 1;
    ++s->events;
    ++s->dropped;
    return KK_OK;
  }
  if (!h_event && !d_event) {
    set_error("kk_stream_push: null event");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(s->device);
  const int g = tu / s->G, j = tu - g * s->G, b = (int)(s->group_seq % s->R);
  cudaError_t e = cudaSuccess;
  if (j == 0 && s->dec_pending[b]) e = cudaStreamWaitEvent(s->s_copy, s->ev_dec[b], 0);  // ring slot free
  if (e == cudaSuccess)
    e = add_copy(s, s->ring[b] + (size_t)j * s->ev_bytes, h_event ? h_event : d_event,
                 h_event ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, extend);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream_push: copy");
  s->next_row = tx_row + 1;
  s->next_tu = tu + 1;
  ++s->events;
  if (j == s->groups[g].n_tx - 1) return run_group(s, g);
  return KK_OK;
}

}  // namespace

extern "C" {

kk_status kk_stream_push_many(kk_stream *s, int32_t first_row, int32_t n_rows, const void *h_events,
                              const void *d_events) {
  if (!s || n_rows < 0) {
    set_error("kk_stream_push_many: null stream or negative count");
    return KK_ERR_INVALID_ARG;
  }
  const unsigned char *h = static_cast<const unsigned char *>(h_events);
  const unsigned char *d = static_cast<const unsigned char *>(d_events);
  for (int32_t r = 0; r < n_rows; ++r) {
    const size_t o = (size_t)r * s->ev_bytes;
    const kk_status st = push_event(s, first_row + r, h ? h + o : nullptr, (!h && d) ? d + o : nullptr, r > 0);
    if (st != KK_OK) return st;
  }
  return KK_OK;
}

kk_status kk_stream_end_frame(kk_stream *s, void *d_B, float *d_I) {
  NvtxRange range("kk_stream_end_frame");
  if (!s) {
    set_error("kk_stream_end_frame: null stream");
    return KK_ERR_INVALID_ARG;
  }
  const kk_plan &p = *s->plan;
  if (s->next_tu != p.Nu) {
    set_error("kk_stream_end_frame: frame incomplete (" + std::to_string(s->next_tu) + " of " +
              std::to_string(p.Nu) + " transmits in use pushed)");
    return KK_ERR_INVALID_ARG;
  }
  if (!d_B || (p.compound != KK_COMPOUND_NONE && !d_I)) {
    set_error("kk_stream_end_frame: null image (or intensity with compounding)");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(s->device);
  const int f = (int)(s->frame % 2);
  cudaError_t e = cudaEventRecord(s->ev_frame_dec[f], s->s_dec);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_img, s->ev_frame_dec[f], 0);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream_end_frame: event");
  const kk_status st = enqueue_beamform(&p, s->rt[f], d_B, d_I, s->ws[f], s->s_img);
  if (st != KK_OK) return st;
  e = cudaEventRecord(s->ev_img[f], s->s_img);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream_end_frame: event");
  s->img_pending[f] = true;
  ++s->frame;
  s->next_row = 0;
  s->next_tu = 0;
  return KK_OK;
}

kk_status kk_stream_wait(kk_stream *s, void *stream) {
  if (!s) {
    set_error("kk_stream_wait: null stream");
    return KK_ERR_INVALID_ARG;
  }
  if (s->frame == 0) return KK_OK;
  DeviceGuard guard(s->device);
  const cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, s->ev_img[(s->frame - 1) % 2], 0);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "kk_stream_wait");
}

kk_status kk_stream_after(kk_stream *s, void *stream) {
  if (!s) {
    set_error("kk_stream_after: null stream");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(s->device);
  cudaError_t e = cudaEventRecord(s->ev_ext, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_img, s->ev_ext, 0);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "kk_stream_after");
}

kk_status kk_stream_sync(kk_stream *s) {
  if (!s) {
    set_error("kk_stream_sync: null stream");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(s->device);
  cudaError_t e = cudaStreamSynchronize(s->s_copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_dec);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_img);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream_sync");
  int32_t v = 0;
  e = cudaMemcpy(&v, s->plan->t.status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "kk_stream_sync: status read");
  if (v != KK_OK) {
    set_error("kk_stream_sync: a bounded device wait gave up");
    return KK_ERR_TIMEOUT;
  }
  return KK_OK;
}

kk_status kk_stream_get_info(const kk_stream *s, kk_stream_info *info) {
  if (!s || !info) {
    set_error("kk_stream_get_info: null argument");
    return KK_ERR_INVALID_ARG;
  }
  info->group = s->G;
  info->ring_groups = s->R;
  info->n_groups = s->n_groups;
  info->events_pushed = s->events;
  info->events_dropped = s->dropped;
  info->groups_run = s->groups_run;
  info->frames_done = s->frame;
  info->device_bytes = s->block_bytes;
  info->copies = s->copies;
  return KK_OK;
}

void kk_stream_destroy(kk_stream *s) {
  if (!s) return;
  DeviceGuard guard(s->device);
  delete s;
}

}  // extern "C"
