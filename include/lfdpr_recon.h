/*
 * lfdpr_recon.h — learned angular reconstruction on top of liblfdpr.so.
 *
 * A display frame can be rendered for a quarter of its views and the rest
 * predicted: LFDPR (lfdpr.h) renders n views (a display with n_views = n over
 * the same cone puts its eyes midway between output views 4j+1 and 4j+2 of
 * the 4n-view display), and a small U-Net predicts the 4n views of the full
 * display after angular supersampling and reconstruction (Sec. 4's 2x
 * angular rate with the [1/4, 1/2, 1/4] tent). The full render is its
 * fallback and the ground truth its error is measured against.
 *
 * Network (fixed architecture, weights supplied by the caller): input = the n
 * views' RGB / 255 as 3n channels (zero padded to 48), views padded with zeros
 * to multiples of 8 pixels; four levels of two 3x3 convolutions + bias + ReLU
 * (channels 32, 64, 128, 256), 2x2 average pooling down, nearest 2x
 * upsampling concatenated with the level's features (upsampled first) up;
 * then a 1x1 convolution to 3 * 4n channels added to the base, clamped to
 * [0, 1], times 255, rounded half to even. The base is the input views
 * warped to the output eyes by their depth keys (lfdpr_warp_views below),
 * RGB / 255 as bf16. Activations and weights are bf16 with fp32
 * accumulation on the tensor cores (tcgen05.mma, accumulators in tensor
 * memory, operands staged by TMA); the 1x1 layer's epilogue adds the base.
 * Activations are held as images with a one-pixel ring of zeros (the 3x3
 * padding), channels in chunks of eight.
 *
 * 3x3 layers in order, (input channels, output channels):
 *   (48,32) (32,32) | (32,64) (64,64) | (64,128) (128,128) | (128,256) (256,256)
 *   | (384,128) (128,128) | (192,64) (64,64) | (96,32) (32,32)
 * Weight blob (bf16 as uint16): each 3x3 layer's [out][3][3][in] in order,
 * then the 1x1 layer's [3 * 4n][32]. Bias blob (f32): each layer's [out] in
 * the same order, then the 1x1 layer's [3 * 4n].
 *
 * Conventions as in lfdpr.h (status codes, lfdpr_last_error, streams).
 */
#ifndef LFDPR_RECON_H
#define LFDPR_RECON_H

#include "lfdpr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lfdpr_recon lfdpr_recon;

/* Number of weights and biases for n input views (the blob sizes above). */
int64_t lfdpr_recon_weight_count(int32_t in_views);
int64_t lfdpr_recon_bias_count(int32_t in_views);

/*
 * lfdpr_create_recon: a network for in_views (even, 2..16) input views of
 * view_w x view_h pixels (8..4032 wide, 8..4096 high); weights_bf16 and biases (host)
 * are copied; the activation buffers are allocated once here.
 * Errors: EINVAL (counts not as above), ENOMEM, ECUDA.
 */
lfdpr_status lfdpr_create_recon(int32_t view_w, int32_t view_h, int32_t in_views, const uint16_t *weights_bf16,
                                int64_t n_weights, const float *biases, int64_t n_biases, lfdpr_recon **out);
lfdpr_status lfdpr_destroy_recon(lfdpr_recon *recon);

/*
 * lfdpr_recon_run: predict the views of display `dst` (4 in_views rendered
 * views, no angular supersampling, same view size) from the rendered views
 * and depth keys of display `src` (in_views rendered views, the last frame
 * rendered), asynchronously on `stream`. The
 * result is in dst's view buffer (lfdpr_get_buffers), so lfdpr_interleave(dst,
 * ...) builds its panel. One network runs one forward pass at a time.
 */
lfdpr_status lfdpr_recon_run(lfdpr_recon *recon, const lfdpr_display *src, lfdpr_display *dst, void *stream);

/* The same on raw device buffers: in_views u8 [in_views][H][W][4], their
 * depth keys in_keys u64 [in_views][H][W], the input and output eyes' x
 * (f32 [in_views], ascending, and [4 in_views]), pixels_per_unit = view_w /
 * focal_w, out_views u8 [4 in_views][H][W][4]. */
lfdpr_status lfdpr_recon_forward(lfdpr_recon *recon, const uint8_t *in_views, const uint64_t *in_keys,
                                 const float *in_eyes, const float *out_eyes, float pixels_per_unit,
                                 uint8_t *out_views, void *stream);

/*
 * lfdpr_recon_status: the failed-wait flags the network's kernels recorded
 * since the last call (0 = none; bit 0: a copy never landed, bit 1: a stage
 * never arrived at the MMA thread, bit 2: the accumulators never completed;
 * each such wait gives up after one second and its block still returns).
 * Synchronous: waits for the device, then clears the flags.
 */
lfdpr_status lfdpr_recon_status(lfdpr_recon *recon, int32_t *flags);

/*
 * lfdpr_warp_views: the depth-guided warp of rendered views to other eyes on
 * the same eye line. Every eye lies on y = 0, z = D and every view shares the
 * focal rectangle at z = 0, so a surface point keeps its pixel row in every
 * view: seen at pixel centre x + 1/2 with ray parameter t from eye E_a (the
 * depth key's high word), it is at x + 1/2 + (1 - 1/t) pixels_per_unit (E -
 * E_a) from eye E (Sec. 3.2's projection through the shared focal plane).
 * For each output eye, the two input views bracketing it (weight s towards
 * the second, clamped to [0, 1]) are moved there: each input pixel with a
 * key lands at pixel floor(x'), the smallest t winning (then the first input,
 * then the leftmost source); a pixel with a winner blends the two inputs,
 * each interpolated linearly along the row at the winner's position in it
 * and counted only where its own key there is within 1 % of the winner's t,
 * with weights (1 - s, s) renormalised by the reciprocal of their sum
 * (neither agreeing: the winner's own source pixel); a pixel with no winner takes (1 - s) c_0 + s c_1 of the
 * inputs at the same pixel. Rounded half to even to RGBA8, alpha 255.
 *  in_views   device u8 [in_count][view_h][view_w][4]
 *  in_keys    device u64 [in_count][view_h][view_w]: the views' depth keys
 *             (lfdpr_get_buffers), all ones where a pixel is empty
 *  in_eyes    device f32 [in_count]: the input eyes' x, ascending
 *  out_eyes   device f32 [out_count]: the output eyes' x
 *  pixels_per_unit  view_w / focal_w of the display
 *  out_views  device u8 [out_count][view_h][view_w][4], caller-owned
 * Limits: 2 <= in_count, 1 <= out_count, both <= 512; view_w <= 4032,
 * view_h <= 16384; views and eyes 4-byte aligned, keys 8-byte aligned.
 * Asynchronous on `stream`. Errors: EINVAL (also a limit or alignment not
 * met), ECUDA.
 */
lfdpr_status lfdpr_warp_views(const uint8_t *in_views, const uint64_t *in_keys, const float *in_eyes, int32_t in_count,
                              const float *out_eyes, int32_t out_count, int32_t view_w, int32_t view_h,
                              float pixels_per_unit, uint8_t *out_views, void *stream);

/*
 * lfdpr_conv3x3_bf16: one 3x3 layer of the network (test hook): in bf16
 * [H][W][cin], wgt bf16 [cout][3][3][cin], bias f32 [cout], out bf16
 * [H][W][cout]: zero padding 1, + bias, ReLU, on the network's tensor-core
 * kernel (the hook converts to and from the network's activation layout).
 * cin % 16 == 0 (<= 512), cout % 32 == 0 (<= 256); device buffers, 16-byte
 * aligned; status: a device int32 that receives the failed-wait flags
 * (OR-ed in, as lfdpr_recon_status describes). Asynchronous on `stream`.
 */
lfdpr_status lfdpr_conv3x3_bf16(const void *in, int32_t H, int32_t W, int32_t cin, const void *wgt,
                                const float *bias, void *out, int32_t cout, int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LFDPR_RECON_H */
