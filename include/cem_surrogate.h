/*
 * cem_surrogate.h -- C ABI of the crack-map surrogate's kernels (libcem.so).
 *
 * The surrogate learns the map from a notched-plate run's inputs -- the
 * traction, the notch and the critical energy release rate field G_c of the
 * explicit solver (include/cem.h) -- to the run's cracked-element map at the
 * end time.  It is a U-Net (levels set by the caller): per level two 3x3
 * convolutions with ReLU, 2x2 max pooling down, nearest 2x upsampling and
 * channel concatenation of the skip up, a 1x1 head to one logit per element,
 * and a class-weighted binary cross-entropy (optionally plus a soft Dice
 * term), trained with Adam.  The paper has no
 * such network; the solver's runs supply its training data.
 *
 * Conventions:
 *   - Activations are BF16 (stored as uint16), NHWC: pixel p = (b*H + h)*W + w,
 *     channel c at p*ld + c, with a pixel stride ld >= C so that a tensor
 *     can be a channel slice of a wider one (concatenation without copies).
 *   - 3x3 weights are [Cout][3][3][Cin] (k = (ky*3 + kx)*Cin + c); BF16
 *     copies feed the tensor cores, FP32 masters receive the updates.
 *   - Accumulation is FP32.  Every reduction adds partial sums in a fixed
 *     order, so results are reproducible run to run.
 *   - All pointers are device memory owned by the caller; `stream` is a
 *     cudaStream_t (NULL = legacy default stream); calls only enqueue work.
 *   - Return 0 (CEM_SG_OK), CEM_SG_ERR_ARG for bad sizes, alignment (channel
 *     counts, strides and offsets of BF16 tensors must be multiples of 8
 *     where stated) or a short workspace, CEM_SG_ERR_CUDA for a failed launch.
 */
#ifndef CEM_SURROGATE_H
#define CEM_SURROGATE_H

#ifdef __cplusplus
extern "C" {
#endif

#define CEM_SG_OK 0
#define CEM_SG_ERR_ARG -1
#define CEM_SG_ERR_CUDA -2

/* y[p, yoff + o] = act(bias[o] + sum_{ky,kx,c} x[p + (ky-1, kx-1), c] w[o][ky][kx][c]),
 * zero outside the image, act = ReLU when relu != 0, and set to zero where
 * mask[p, o] <= 0 when mask (pixel stride ldmask) is given -- the data
 * gradient of a layer whose input is a ReLU output.  Cin, ldx multiples of 8;
 * Cout, yoff, ldmask even; bias, mask may be NULL.  Implicit GEMM on the
 * tensor cores. */
int cem_sg_conv3x3(const void *x, int B, int H, int W, int Cin, int ldx, const void *w,
                   const float *bias, int Cout, int relu, const void *mask, int ldmask, void *y,
                   int ldy, int yoff, void *stream);

/* Workspace bytes cem_sg_conv3x3_wgrad needs for this shape. */
long cem_sg_wgrad_workspace(int B, int H, int W, int Cin, int Cout);

/* Weight and bias gradients of the 3x3 convolution: dw[o][ky][kx][c] =
 * sum_p dy[p, o] x[p + (ky-1, kx-1), c] (FP32), db[o] = sum_p dy[p, o]
 * (db may be NULL).  The data gradient is cem_sg_conv3x3 applied to dy with
 * the transposed, flipped weights that cem_sg_adam writes.  Cin, Cout, ldx,
 * lddy multiples of 8. */
int cem_sg_conv3x3_wgrad(const void *x, int ldx, const void *dy, int lddy, int B, int H, int W,
                         int Cin, int Cout, float *dw, float *db, void *ws, long ws_bytes,
                         void *stream);

/* dy[p, c] = 0 where y[p, c] <= 0, p < P, c < C (pixel strides lddy, ldy):
 * gradient through ReLU given its output. */
int cem_sg_relu_bwd(void *dy, int lddy, const void *y, int ldy, long P, int C, void *stream);

/* 2x2 max pooling of x [B, 2H, 2W] (pixel stride ldx, channels 0..C-1) into
 * dense y [B, H, W, C].  Pooling and upsampling need C, strides and channel
 * offsets that are multiples of 8 (16-byte vectors). */
int cem_sg_maxpool2(const void *x, int ldx, int B, int H, int W, int C, void *y, void *stream);

/* Its gradient: dy [B, H, W, C] goes to the first maximum (window order
 * (0,0), (0,1), (1,0), (1,1)) of each window of x; dskip (channels skoff ..
 * skoff+C-1 of a [B, 2H, 2W, ldskip] tensor, may be NULL) is added; with
 * relu_mask the result is zero where x <= 0 (x a ReLU output); dx is dense
 * [B, 2H, 2W, C]. */
int cem_sg_maxpool2_bwd(const void *x, int ldx, const void *dy, const void *dskip, int ldskip,
                        int skoff, int B, int H, int W, int C, int relu_mask, void *dx,
                        void *stream);

/* Nearest 2x upsampling of dense x [B, H, W, C] into channels yoff ..
 * yoff+C-1 of y [B, 2H, 2W, ldy]. */
int cem_sg_upsample2(const void *x, int B, int H, int W, int C, void *y, int ldy, int yoff,
                     void *stream);

/* Its gradient: dx [B, H, W, C] = sum of each 2x2 block of dy's channels
 * 0..C-1 (dy [B, 2H, 2W, lddy]), zero where mask [B, H, W, ldmask] <= 0
 * when mask is given (the upsampled tensor a ReLU output). */
int cem_sg_upsample2_bwd(const void *dy, int lddy, int B, int H, int W, int C, const void *mask,
                         int ldmask, void *dx, void *stream);

/* 1x1 head: z[p] = b[0] + sum_c x[p, c] w[c] (FP32 logits, x dense [P, C]). */
int cem_sg_head_fwd(const void *x, int P, int C, const float *w, const float *b, float *z,
                    void *stream);

long cem_sg_head_workspace(int P, int C);

/* Its gradients: dx[p, c] = dz[p] w[c] where x[p, c] > 0, else 0 (x is a
 * ReLU output; BF16), dw[c] = sum_p dz[p] x[p, c], db[0] = sum_p dz[p].
 * C <= 32. */
int cem_sg_head_bwd(const void *x, int P, int C, const float *w, const float *dz, void *dx,
                    float *dw, float *db, void *ws, long ws_bytes, void *stream);

long cem_sg_bce_workspace(long n);

/* Class-weighted binary cross-entropy with logits, mean over n elements:
 * loss = mean(pw t log(1 + e^-z) + (1 - t) log(1 + e^z)), t in {0, 1}
 * (uint8), and dz = d loss / d z. */
int cem_sg_bce(const float *z, const unsigned char *t, long n, float pos_weight, float *dz,
               float *loss, void *ws, long ws_bytes, void *stream);

/* Workspace bytes cem_sg_dice needs (0 for bad sizes). */
long cem_sg_dice_workspace(int B, long n_per);

/* Soft Dice loss of B samples of n_per logits each (z, t sample-major,
 * t in {0, 1}), weighted by `weight`: with p = sigmoid(z), per sample
 * D_b = (2 sum p t + eps) / (sum p + sum t + eps), and
 *   loss[0] = weight (1 - mean_b D_b)       (overwritten),
 *   dz     += weight d(1 - mean_b D_b)/dz   (added, e.g. to the BCE gradient).
 * The overlap of the predicted and the target cracked sets is what the
 * surrogate is judged by (the Jaccard index J = D / (2 - D) on hard maps);
 * this term trains for it directly.  eps > 0; sums in a fixed order. */
int cem_sg_dice(const float *z, const unsigned char *t, int B, long n_per, float weight, float eps,
                float *dz, float *loss, void *ws, long ws_bytes, void *stream);

/* One Adam step (Kingma and Ba, bias-corrected, step >= 1) on n FP32
 * weights w with gradient g and moments m, v; writes the BF16 copy w_bf16
 * (may be NULL) and, for 3x3 weights (n = Cout*9*Cin), the transposed,
 * flipped BF16 copy wt_bf16[c][ky][kx][o] = w[o][2-ky][2-kx][c] used by the
 * data gradient (may be NULL).  lr = 0 only refreshes the copies (with the
 * moments still advanced). */
int cem_sg_adam(float *w, const float *g, float *m, float *v, long n, float lr, float beta1,
                float beta2, float eps, int step, void *w_bf16, void *wt_bf16, int Cout, int Cin,
                void *stream);

/* Selects the tensor-core path of cem_sg_conv3x3 for later calls: 1 (the
 * default) = tcgen05 MMAs with a TMEM accumulator and a 2-stage
 * shared-memory ring (CTAs of 128 threads, two to five per SM), 0 = warp-level mma.sync
 * m16n8k16 with register accumulators.  Both compute the same sums (FP32
 * accumulation in a different order).  Process-wide; not synchronised with
 * work in flight. */
int cem_sg_set_gemm_path(int use_tcgen05);

/* Number of tcgen05 CTAs whose bounded wait for their MMAs gave up since the
 * library was loaded (0 in a healthy run).  Such a CTA leaves its output
 * tile unwritten, waits (bounded) for the MMAs it had issued, and frees its
 * tensor memory only if they finished: the results of any call during which
 * the count grew are invalid, and the binding's training and inference
 * check the count around each epoch and evaluation and fail when it grows.
 * Synchronises with the device. */
int cem_sg_timeouts(int *count);

/* y = BF16(x), n elements. */
int cem_sg_to_bf16(const float *x, long n, void *y, void *stream);

#ifdef __cplusplus
}
#endif
#endif
