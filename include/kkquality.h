/*
 * kkquality.h -- C ABI of the image-quality measures used to judge KK and
 * DAS images: the generalized contrast-to-noise ratio (gCNR) of an inclusion
 * against a background region, and the half-amplitude widths (FWHM) of point
 * targets.  The paper judges contrast by gCNR (Section III, Fig. 5; the
 * measure is defined in the references its Experimental Methods paragraph
 * cites) and resolution by the width and separability of wire targets
 * (Section III, Fig. 4).
 *
 * Definitions (every integer below is decided in the stated precision, so
 * two implementations that follow them agree exactly):
 *  - envelope e = |B| of a complex image, or sqrt(I) of an intensity image,
 *    formed in float32 with one IEEE rounding per operation (re*re, im*im,
 *    their sum, the square root; no fused multiply-add).
 *  - a pixel belongs to a region when its centre (x0 + ix*dx, z0 + iz*dz),
 *    computed in float64 with one rounding per operation, satisfies
 *      disk     (a, b) = centre, c = r:         (x-a)^2 + (z-b)^2 <= c^2
 *      annulus  (a, b) = centre, c < d radii:   c^2 < (x-a)^2 + (z-b)^2 <= d^2
 *      rect     [a, b] x [c, d] (x then z):    a <= x <= b and c <= z <= d
 *    (squares and sums in float64, one rounding each).
 *  - gCNR = 1 - sum_b min(p_in[b], p_out[b]), p = bin counts / region size,
 *    over n_bins equal-width bins spanning [lo, hi], the envelope range over
 *    both regions.  A value v falls in bin floor(((v - lo) * n_bins) /
 *    (hi - lo)) computed in float32 (one rounding per operation), clamped to
 *    n_bins - 1; hi == lo puts every value in bin 0.  The overlap is summed
 *    exactly in integers, sum_b min(c_in[b] * n_out, c_out[b] * n_in), and
 *    divided once by n_in * n_out in float64.  An empty region gives NaN.
 *  - FWHM: the first maximum of e in row-major order inside the target's
 *    search window [ix-wx, ix+wx] x [iz-wz, iz+wz] (clipped to the image);
 *    along the peak's row (lateral) and column (axial), on each side the
 *    nearest sample strictly below half the peak (half = 0.5 * peak in
 *    float32); the crossing lies between it and its inner neighbour by linear
 *    interpolation in float64; the width is the distance between the two
 *    crossings in metres.  A side that reaches the image edge first gives a
 *    NaN width; an empty window gives ix = iz = -1 and NaN everywhere.
 *
 * Layouts: a batch of images is [n_images][nz][nx], cfloat (interleaved re,
 * im float32, as kk_beamform writes B) or float32 (as kk_beamform writes I).
 * Inputs must be finite.
 *
 * Conventions as in kkbeam.h: device pointers unless stated, calls that take
 * a stream only enqueue (no allocation, no synchronisation: they may be
 * captured in a CUDA graph), errors are kk_status with kk_last_error().
 */
#ifndef KKQUALITY_H
#define KKQUALITY_H

#include "kkbeam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kk_region_kind {
  KK_REGION_DISK = 0,
  KK_REGION_ANNULUS = 1,
  KK_REGION_RECT = 2
} kk_region_kind;

typedef enum kk_image_kind {
  KK_IMAGE_COMPLEX = 0,   /* cfloat B, envelope |B| */
  KK_IMAGE_INTENSITY = 1  /* float32 I, envelope sqrt(I) */
} kk_image_kind;

/* A region of the image plane (metres); parameters as described above. */
typedef struct kk_region {
  int32_t kind; /* kk_region_kind */
  double a, b, c, d;
} kk_region;

/* A point target: search window centre (ix, iz) and half-widths (wx, wz),
 * all in pixels; wx, wz >= 0. */
typedef struct kk_target {
  int32_t ix, iz, wx, wz;
} kk_target;

/* Result of one (image, target): peak pixel, peak envelope, widths in
 * metres (NaN where undefined). */
typedef struct kk_fwhm_result {
  int32_t ix, iz;
  float peak;
  int32_t reserved;
  double lateral, axial;
} kk_fwhm_result;

typedef struct kk_quality_desc {
  kk_grid grid;               /* shared by every image; nx, nz >= 1, dx, dz > 0 */
  int32_t image_kind;         /* kk_image_kind */
  int32_t n_contrast;         /* >= 0 (inside, outside) region pairs */
  const kk_region *inside;    /* host [n_contrast] */
  const kk_region *outside;   /* host [n_contrast] */
  int32_t n_bins;             /* 1..4096 */
  int32_t n_targets;          /* >= 0 */
  const kk_target *targets;   /* host [n_targets] */
  int32_t device;             /* CUDA device ordinal */
} kk_quality_desc;

typedef struct kk_quality kk_quality;

/* Validates the description, copies the regions and targets and builds each
 * region pair's pixel labels on the device (synchronous).  Regions may lie
 * partly or wholly outside the grid.  KK_ERR_INVALID_ARG for a bad size,
 * kind or non-finite parameter; KK_ERR_OOM / KK_ERR_CUDA from the device. */
kk_status kk_quality_create(kk_quality **out, const kk_quality_desc *d);
void kk_quality_destroy(kk_quality *q);

/* gcnr[n][m] = gCNR of image n for region pair m; d_gcnr is float64
 * [n_images][n_contrast] on the device.  n_images >= 0 (0: nothing). */
kk_status kk_quality_gcnr(const kk_quality *q, const void *d_images, int32_t n_images,
                          double *d_gcnr, void *stream);

/* out[n][t] = FWHM result of image n for target t; d_out is
 * [n_images][n_targets] on the device.  n_images >= 0 (0: nothing). */
kk_status kk_quality_fwhm(const kk_quality *q, const void *d_images, int32_t n_images,
                          kk_fwhm_result *d_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KKQUALITY_H */
