/*
 * kkstream.h -- C ABI of the streaming decomposition: the far-field
 * decomposition of Eq. (compression) applied to each group of transmit
 * events as the events arrive, overlapped with the image formation, Eq. (KK),
 * of the previous frame.
 *
 * The paper performs the decomposition in software after the whole
 * acquisition, and names doing it in hardware as the data arrives (in the
 * probe, Section IV) as a way to cut the data moved to the host.  This is
 * that scheme on one GPU:
 *   - transmit events (one transmit angle's channel data, [L][T] samples)
 *     are pushed in acquisition order; events of transmits the plan does not
 *     use are dropped without a copy;
 *   - each event is copied into a device ring of R groups of G events (events
 *     contiguous in both the source and the ring share one copy, issued when
 *     the group fills), so
 *     copies may run up to R - 1 groups ahead of the decomposition; when a
 *     group is complete its spectrum, contraction and inverse run on
 *     the decomposition stream and write that group's pairs into the frame's
 *     rf_theta;
 *   - when the frame's last used transmit has been pushed, kk_stream_end_frame
 *     runs the image formation of the frame on the image stream, reading one
 *     of two rf_theta buffers while the next frame's groups fill the other.
 * Every dependency (a ring slot free again, a group copied, an rf_theta
 * buffer free again, a frame decomposed) is a CUDA event between the
 * stream's three CUDA streams; no kernel waits on another, so nothing spins.
 * Results equal those of kk_decompose + kk_beamform on the whole frame (the
 * same kernels, per group of transmits).
 *
 * Conventions as in kkbeam.h: calls only enqueue (except create and sync),
 * errors are kk_status with kk_last_error().
 */
#ifndef KKSTREAM_H
#define KKSTREAM_H

#include "kkbeam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kk_stream kk_stream;

typedef struct kk_stream_info {
  int32_t group;            /* transmit events per decomposition group */
  int32_t ring_groups;      /* R: groups the device ring holds */
  int32_t n_groups;         /* groups per frame: ceil(transmits in use / group) */
  int64_t events_pushed;    /* all pushed events */
  int64_t events_dropped;   /* of which: transmits the plan does not use */
  int64_t groups_run;       /* decomposition groups enqueued */
  int64_t frames_done;      /* frames whose image formation is enqueued */
  size_t device_bytes;      /* ring, scratch, two rf_theta buffers, two workspaces */
  int64_t copies;           /* host-to-device copies issued (events contiguous in
                               both source and ring share one copy) */
} kk_stream_info;

/* Creates a stream for a KK plan (not DAS), with `group` transmit events per
 * decomposition group, 1 <= group <= transmits in use, and a device ring of
 * ring_groups groups, 2 <= ring_groups <= 64 (a frame's worth plus one lets
 * every copy of the next frame land while the current frame is imaged).
 * Allocates its device buffers and three CUDA streams (decomposition and
 * copies at high priority).  The plan must outlive the stream.  Synchronous. */
kk_status kk_stream_create(kk_stream **out, const kk_plan *plan, int32_t group, int32_t ring_groups);

/* Pushes the transmit event of row tx_row (0 <= tx_row < the plan's n_tx),
 * [L][T] samples of the plan's rf dtype.  Within a frame rows must increase;
 * a row the plan uses may not be skipped.  h_event is host memory (pinned
 * for an asynchronous copy; it must stay unchanged until kk_stream_sync or
 * until the group containing it has been decomposed); d_event (used when
 * h_event is NULL) is device memory with the same lifetime rule.  Returns
 * KK_ERR_INVALID_ARG for an out-of-order or skipped row and for a push after
 * the frame is complete. */
kk_status kk_stream_push(kk_stream *s, int32_t tx_row, const void *h_event, const void *d_event);

/* Pushes rows first_row .. first_row + n_rows - 1 from one block of
 * consecutive events, [n_rows][L][T] at h_events (host) or d_events (device,
 * used when h_events is NULL); the same rules as kk_stream_push, event by
 * event.  An error leaves the rows before the failing one pushed. */
kk_status kk_stream_push_many(kk_stream *s, int32_t first_row, int32_t n_rows, const void *h_events,
                              const void *d_events);

/* Ends the current frame (all transmits in use pushed): enqueues its image
 * formation into d_B [J][nz][nx] cfloat and d_I [nz][nx] (required when the
 * plan compounds, else nullable), as kk_beamform does.  The outputs are
 * complete when kk_stream_sync returns or after kk_stream_wait on a caller
 * stream.  KK_ERR_INVALID_ARG if the frame is incomplete. */
kk_status kk_stream_end_frame(kk_stream *s, void *d_B, float *d_I);

/* Makes `stream` (a cudaStream_t) wait for the last ended frame's image. */
kk_status kk_stream_wait(kk_stream *s, void *stream);

/* Makes the image formations enqueued from now on wait for the work already
 * enqueued on `stream` (a cudaStream_t): e.g. the download of an earlier
 * frame's B and I before those buffers are passed to kk_stream_end_frame
 * again. */
kk_status kk_stream_after(kk_stream *s, void *stream);

/* Waits for all enqueued work; returns the plan's device status
 * (KK_ERR_TIMEOUT if a bounded device wait gave up, else KK_OK). */
kk_status kk_stream_sync(kk_stream *s);

kk_status kk_stream_get_info(const kk_stream *s, kk_stream_info *info);

/* Synchronises, then frees the stream's buffers and CUDA streams. */
void kk_stream_destroy(kk_stream *s);

#ifdef __cplusplus
}
#endif

#endif /* KKSTREAM_H */
