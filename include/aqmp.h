/*
 * aqmp.h -- C ABI of the GB300 (sm_103a) AQMP encoder library, libaqmp.so.
 *
 * AQMP (Adaptive Quadtree Matching Pursuit) encodes each image plane by
 * Matching Pursuit over the blocks of a quadtree: a block that misses the
 * accuracy tolerance within its atom budget is split into four quadrants
 * that restart from the original pixels (Section 2.3, Algorithms 1-2); a
 * decoder rebuilds the plane as y = D_N x per leaf (Algorithm 3).
 *
 * Conventions shared by every entry point:
 *   - Return 0 (AQMP_OK) or a negative AQMP_E_* code; aqmp_last_error()
 *     then holds a one-line message for the calling thread.
 *   - Pointers are plain host or device addresses as stated per argument;
 *     nothing here takes ownership of caller memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; calls that return counts synchronise it first.
 *   - There is no CPU fallback: without a usable sm_103a GPU every call that
 *     computes returns AQMP_E_CUDA.
 */
#ifndef AQMP_H
#define AQMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AQMP_OK                 0
#define AQMP_E_ARG             -1  /* NULL pointer, bad block sizes or parameters */
#define AQMP_E_SHAPE           -2  /* plane size not a multiple of max_block */
#define AQMP_E_DICT            -3  /* unknown dictionary id */
#define AQMP_E_OOM             -4  /* device or host allocation failed */
#define AQMP_E_CUDA            -5  /* CUDA runtime / driver error, or no usable GPU */
#define AQMP_E_QUEUE_OVERFLOW  -6  /* a device work queue or output ran out of room */
#define AQMP_E_TIMEOUT         -7  /* a bounded device wait gave up */
#define AQMP_E_UNSUPPORTED     -8  /* valid request this build does not serve */

/* Dictionaries (Section 2.3 / Appendix A: a DCT basis concatenated with
 * Haar wavelets).  At block side b the atoms are the b^2 2-D DCT-II atoms
 * (Section 2.1, Eq. (1)-(2), outer products of 1-D rows) followed by the b^2
 * 2-D Haar atoms; the single-family dictionaries exist for testing. */
#define AQMP_DICT_DCT_HAAR  0      /* M = 2 b^2 atoms */
#define AQMP_DICT_DCT       1      /* M = b^2 */
#define AQMP_DICT_HAAR      2      /* M = b^2 */

/* Arithmetic of the pursuit (see aqmp_params.precision). */
#define AQMP_PREC_EXACT     0      /* exact-limb BF16 tensor-core correlation +
                                      double-float pursuit: decisions agree with
                                      an FP64 evaluation except where a
                                      decision margin is below ~2^-36 of the
                                      block norm, and such leaves are flagged */
#define AQMP_PREC_FP32      1      /* the plain FP32 form: the same correlation
                                      rounded to FP32, FP32 pursuit state (one
                                      FMA per Gram entry), FP32 energy and stop
                                      test; faster, decisions not certified */
#define AQMP_PREC_BF16      2      /* the reduced-precision form: the correlation
                                      from one BF16 tensor-core pass of bf16(D)
                                      (FP32 accumulation, no exact digits), then
                                      the FP32 form's pursuit; decisions not
                                      certified */
#define AQMP_PREC_FP8       3      /* the FP8 form: one E4M3 tensor-core pass
                                      (kind::f8f6f4) of e4m3(D s_j) against
                                      e4m3((y - 128) s_l), s_j and s_l powers of
                                      two per atom and per block (the largest
                                      keeping the values within 448), FP32
                                      accumulation, rescaled; then the FP32
                                      form's pursuit; decisions not certified */
#define AQMP_PREC_BF16_RESCORE 4   /* the BF16 form with rescore: at side 64 the
                                      correlation from split BF16 tensor-core
                                      products of the separable form, with a
                                      per-atom error bound
                                      (aqmp_correlate_bf16x2); the exact form's
                                      pursuit, in which every atom that could
                                      be the argmax under those bounds first
                                      gets its exact initial correlation
                                      recomputed from the pixels (at most 8 per
                                      step; a leaf needing more is redone by the
                                      exact form); decisions certified as in
                                      the exact form.  Other sides: the exact
                                      form.  Needs the DCT+Haar dictionary or a
                                      single family, any max_block. */

/* aqmp_params.flags */
#define AQMP_FLAG_INPUT_DEVICE  1u /* plane pointers are device addresses */
#define AQMP_FLAG_SIMT_GEMM     2u /* compute the initial correlation with the
                                      integer SIMT kernel instead of tcgen05
                                      (bit-identical result; for validation) */
#define AQMP_FLAG_NO_AUTOTUNE   4u /* use the default kernel at every side instead
                                      of the autotuned choice */
#define AQMP_FLAG_ALT_THREADS   8u /* run the pursuit with its alternate launch
                                      shape: the other threads per leaf at
                                      sides 16 and 32, two resident CTAs per SM
                                      at side 64 (bit-identical result; for
                                      validation) */
#define AQMP_FLAG_OMP          16u /* Orthogonal Matching Pursuit (the solver the
                                      paper's authors ran, Section 2.2) instead
                                      of MP: after each selection the support's
                                      coefficients are re-fitted by least
                                      squares (FP64 Cholesky); the emitted
                                      coefficients are the final fit.  Needs
                                      max_block <= 64, AQMP_PREC_EXACT and a
                                      budget per leaf of at most 64 atoms at
                                      sides 4..16 and 1024 at sides 32 and 64
                                      (else AQMP_E_UNSUPPORTED).  Sides 32 and
                                      64 keep a Cholesky factor of up to
                                      k(k+1)/2 doubles per SM in device
                                      memory (4.2 MB at k = 1024). */
/* Autotuning: kernel choices that leave the result unchanged bit for bit
 * are measured on the first calls of each configuration and the fastest
 * is kept for the life of the process: the initial correlation on the
 * tensor cores or on the integer SIMT path (both are timed, twice each, on
 * the first encode that meets a side, dictionary, precision and capacity),
 * and the pursuit's launch shape at sides 16, 32 and 64 (threads per leaf,
 * or resident CTAs per SM at side 64; the two candidates alternate over the
 * first four such encodes). */

typedef struct {
    float   rmse_tol;     /* per-block RMSE tolerance on the 0-255 scale:
                             a block converges when ||r||^2 < tol^2 b^2
                             (Eq. (3) with eps = tol b); >= 0 */
    int32_t cap_num;      /* atom budget k(b) = max(1, b^2 cap_num / cap_den) */
    int32_t cap_den;      /*   (min_sparsity of Algorithm 2), cap <= 1 */
    int32_t min_block;    /* N_min, N_max: powers of two, 4 <= N_min <= N_max */
    int32_t max_block;    /*   <= 128 (Section 2.3, set S); a side-128
                             leaf runs on a cluster of four CTAs (two for a
                             single-family dictionary), its correlation on
                             the tensor cores in four exact K chunks */
    int32_t dict_id;      /* AQMP_DICT_* */
    int32_t precision;    /* AQMP_PREC_* */
    uint32_t flags;       /* AQMP_FLAG_* */
} aqmp_params;

/* Default parameters: tol 2, k = b^2/4, blocks 64 -> 4, DCT+Haar, exact. */
void aqmp_params_default(aqmp_params *p);

/* One 8-bit plane to encode (Algorithm 1 processes channels independently;
 * each plane carries its own tolerance so that a batch can sweep it). */
typedef struct {
    const uint8_t *pixels;  /* row-major; host or device per the flags */
    int32_t height;         /* multiples of max_block */
    int32_t width;
    int64_t pitch;          /* bytes between rows, >= width */
    float   rmse_tol;       /* this plane's tolerance; < 0 = params->rmse_tol */
} aqmp_plane;

/* One leaf of the quadtree: block side b at (y, x) of `plane`, owning atoms
 * [atom_off, atom_off + n_atoms) of the atom array. */
typedef struct {
    uint32_t plane;
    uint32_t y, x;
    uint32_t atom_off;
    uint16_t b;
    uint16_t n_atoms;
    uint8_t  converged;     /* 1 if ||r||^2 < eps^2 was reached */
    uint8_t  flags;         /* AQMP_LEAF_* */
    uint16_t reserved;
} aqmp_leaf;

#define AQMP_LEAF_NEAR_TIE        1u  /* a decision of this leaf's pursuit fell
                                         inside the certification band */
#define AQMP_LEAF_NEAR_TIE_PARENT 2u  /* ... or one of an ancestor's (failed)
                                         pursuits did */

/* One MP step: atom index j (DCT atoms 0..b^2-1, Haar atoms b^2..2b^2-1;
 * within a family atom (p, q) has index q b + p) and coefficient alpha.
 * A leaf's atoms are listed in the order the pursuit chose them. */
typedef struct {
    uint32_t j;
    float    alpha;
} aqmp_atom;

/* Work and outcome counters of one encode call. */
typedef struct {
    uint64_t n_leaves;
    uint64_t n_atoms;
    uint64_t attempts;          /* pursuits run, including those that split */
    uint64_t atom_iterations;   /* MP steps run, including those of split blocks */
    uint64_t near_tie_leaves;   /* leaves with any AQMP_LEAF_* flag */
    uint64_t attempts_per_level[8];
    uint64_t iterations_per_level[8];
    uint64_t window_steps_per_level[8];   /* steps decided in full precision because
                                           * another atom lay within the decision
                                           * window of the largest (exact form) */
    uint64_t max_leaf_steps_per_level[8]; /* steps of the level's longest pursuit: the
                                           * level's serial chain (its launch cannot
                                           * end before that pursuit does) */
    uint64_t rescored_atoms;    /* AQMP_PREC_BF16_RESCORE: exact initial
                                 * correlations recomputed */
    uint64_t fallback_leaves;   /* AQMP_PREC_BF16_RESCORE: leaves redone by the
                                 * exact form */
    uint64_t rescore_rounds;    /* AQMP_PREC_BF16_RESCORE: rounds of exact
                                 * recomputation (up to 8 atoms each) */
} aqmp_stats;

typedef struct aqmp_code aqmp_code;   /* opaque, library-owned result */

/* Encode `n_planes` planes (Algorithms 1-2).  Pixels are read on `stream`
 * (copied in first when they are host memory); on success *out receives a
 * new code object whose leaf and atom arrays live in device memory.  The
 * call synchronises `stream` before returning.  Errors: AQMP_E_ARG,
 * AQMP_E_SHAPE, AQMP_E_DICT, AQMP_E_OOM, AQMP_E_CUDA, AQMP_E_QUEUE_OVERFLOW,
 * AQMP_E_TIMEOUT; *out is left NULL on error. */
int aqmp_encode_planes(const aqmp_params *params, const aqmp_plane *planes, int n_planes,
                       void *stream, aqmp_code **out);

/* Convenience form: `channels` planes of h x w stacked one after another,
 * plane c starting at pixels + c h pitch; every plane uses params->rmse_tol. */
int aqmp_encode(const aqmp_params *params, const uint8_t *pixels, int channels, int h, int w,
                size_t pitch, void *stream, aqmp_code **out);

/* Batch form (Algorithm 1 over several images): image i has channels[i]
 * planes of h[i] x w[i] stacked one after another at images[i] (plane c at
 * images[i] + c h[i] pitch[i]); all planes of all images go through one
 * encode, planes numbered image by image, and use params->rmse_tol. */
int aqmp_encode_batch(const aqmp_params *params, int n_images, const uint8_t *const *images,
                      const int *channels, const int *h, const int *w, const size_t *pitch,
                      void *stream, aqmp_code **out);

/* Counters of a finished encode (host struct, filled in place). */
int aqmp_code_stats(const aqmp_code *code, aqmp_stats *stats);

/* Host copies of the result in canonical order: planes ascending, roots
 * row-major, leaves depth-first with children TL, TR, BL, BR.  `leaves`
 * needs stats.n_leaves entries and `atoms` stats.n_atoms; atom_off in the
 * copied leaves indexes the copied atom array.  `alpha_lo`, if not NULL,
 * receives n_atoms floats: the low word of each coefficient as computed
 * (alpha = atoms[i].alpha + alpha_lo[i] to ~2^-48 relative). */
int aqmp_code_copy(const aqmp_code *code, aqmp_leaf *leaves, aqmp_atom *atoms, float *alpha_lo);

/* Decode one plane (Algorithm 3): writes height x width floats, row-major
 * with `out_pitch` elements between rows, into `out` (device memory if
 * out_is_device, else host memory).  Unclipped reconstruction. */
int aqmp_decode(const aqmp_code *code, int plane, float *out, int64_t out_pitch,
                int out_is_device, void *stream);

void aqmp_code_free(aqmp_code *code);

/* ---- Differentiable refinement of the coefficients on a fixed support ----
 * The support (leaves and atom indices) of an encode is held fixed; the
 * coefficients become variables of the synthesis of Algorithm 3 and of the
 * SSIM of Section 3, so that they can be refined by gradient descent.  These
 * calls work on device memory only, in the code's device atom order
 * (aqmp_code_device), and enqueue on `stream` without synchronising. */

/* Device views of an encode: leaf and atom arrays in canonical order (the
 * order the coefficient vectors below follow), and their counts. */
int aqmp_code_device(const aqmp_code *code, const aqmp_leaf **leaves, const aqmp_atom **atoms,
                     uint64_t *n_leaves, uint64_t *n_atoms);

/* Synthesis (Algorithm 3) of one plane with caller coefficients: out[y][x]
 * = sum over the plane's leaves of sum_t alpha[t] phi_{j_t}, where alpha has
 * n_atoms entries (FP32); out is h x w with `out_pitch` elements per row. */
int aqmp_synth_forward(const aqmp_code *code, int plane, const float *alpha, float *out,
                       int64_t out_pitch, void *stream);

/* Its adjoint: grad_alpha[t] = <grad_out restricted to the atom's leaf,
 * phi_{j_t}> for the atoms of `plane` (other entries are left untouched). */
int aqmp_synth_backward(const aqmp_code *code, int plane, const float *grad_out, int64_t pitch,
                        float *grad_alpha, void *stream);

/* Mean SSIM (Section 3; K1 = 0.01, K2 = 0.03, L = 255, 11x11 Gaussian
 * window of sigma 1.5, valid region) of `y` against the reference `x`, both
 * h x w FP32 images with `pitch` elements per row, h, w >= 11.  Window
 * sums are accumulated in double-float (~2^-46 relative), the per-window
 * formula in FP64.  *ssim (device, FP64) receives the
 * mean; with grad_y != NULL, grad_y (h x w, pitch) receives
 * grad_scale * d(mean SSIM)/dy. */
int aqmp_ssim(const float *x, const float *y, int h, int w, int64_t pitch, double *ssim,
              float *grad_y, double grad_scale, void *stream);

/* The initial correlation of Section 2.2 step (b) for a batch of L blocks
 * of side b: c[l][j] = <y_l, phi_j> for every atom j, with y_l the
 * column-major unravel of block l (Appendix A).  `blocks` is device memory
 * holding L blocks of b x b bytes, each row-major and contiguous; `corr` is
 * device memory, 16-byte aligned (else AQMP_E_ARG), for L x M float pairs
 * (hi, lo) whose sum is the correlation of the 2^-48 fixed-point dictionary
 * with the block, rounded once.
 * gemm selects the kernel:
 *   0 = the separable exact correlation B Y B^T: at side 64 the DCT-II
 *       family on tcgen05 and the Haar family on the integer SIMT pipes,
 *       the integer SIMT kernel at the other sides;
 *   1 = the separable SIMT kernel at every side;
 *   6 = the separable tcgen05 kernel for every family, side 64 only (else
 *       AQMP_E_UNSUPPORTED)
 *       (0, 1 and 6 round the same exact integer once: identical bits);
 *   3, 4 = the dense exact kernels (round(D 2^48), tcgen05 and SIMT);
 *   2 = the reduced-precision BF16 form (one tcgen05 pass of bf16(D), FP32
 *       accumulation; low words 0);
 *   5 = the FP8 form (one E4M3 tcgen05 pass, per-atom and per-block
 *       power-of-two scales; low words 0).
 * On a kernel error the stream is synchronised before the error returns. */
int aqmp_correlate(int b, int dict_id, const uint8_t *blocks, int64_t L, float *corr,
                   int gemm, void *stream);

/* The initial correlation of the BF16 form with rescore (the correlation
 * GEMM in BF16 on the tensor cores with FP32 accumulation; Section 2.1, 2-D
 * atoms as outer products of 1-D rows), side 64 only (else
 * AQMP_E_UNSUPPORTED).  For L blocks laid out as for aqmp_correlate:
 * `corr` (device, L x M float pairs) receives c~ ~ B Y B^T per family from
 * split BF16 products of the 1-D rows and of the intermediate, the pixels
 * centred on each block's integer mean; `bound` (device, L x M floats)
 * receives e_j >= |c~_j - c_j|, c_j the value aqmp_correlate (gemm 0)
 * returns, under the accumulation model stated in the kernel's header (each
 * FP32 MMA step errs by at most two units in the last place of its running
 * magnitude). */
int aqmp_correlate_bf16x2(int b, int dict_id, const uint8_t *blocks, int64_t L, float *corr, float *bound,
                          void *stream);

/* Kernel timing.  While enabled, every kernel the library launches is
 * bracketed by CUDA events on the stream it runs on; the durations are
 * folded into per-kernel totals when the launching call synchronises.
 * Names are "<kernel>_b<side>" (e.g. "mp_b64", "corr_tc_b16"). */
typedef struct {
    char     name[32];
    uint64_t launches;
    double   total_ms;
} aqmp_kernel_time;

int  aqmp_profile_enable(int on);                 /* returns the previous state */
void aqmp_profile_reset(void);
/* Copies up to `max` entries into `out` (host); *n receives the count. */
int  aqmp_profile_read(aqmp_kernel_time *out, int max, int *n);
/* Time only the kernels whose name starts with `prefix` (NULL or "": all);
 * each timed launch adds two event records to the stream's timeline. */
int  aqmp_profile_filter(const char *prefix);

/* Autotuner state of the current device (see AQMP_FLAG_NO_AUTOTUNE): one
 * entry per choice point met so far.  kind 0 = initial correlation
 * (candidate 0 tcgen05, 1 integer SIMT); kind 1 = pursuit (candidate 0 the
 * default threads per leaf, 1 the alternate).  chosen is -1 while the
 * candidates are still being timed; best_ms is each candidate's lowest
 * timing.  Copies up to `max` entries into `out`; *n receives the count. */
typedef struct {
    int    kind, side, dict_id, precision, capacity_log2;
    int    chosen;
    int    samples[2];
    double best_ms[2];
} aqmp_tune_entry;

int  aqmp_autotune_read(aqmp_tune_entry *out, int max, int *n);
void aqmp_autotune_reset(void);   /* forget every choice (they are measured again) */

/* aqmp_correlate without any device allocation, for callers that may not
 * allocate device memory (memory owned by another allocator or by a fixed
 * budget, loops that reserve everything at start-up).  The paper has no
 * counterpart: this is a deployment variant of the correlation above; it
 * takes the same arguments except the kernel choice (it always runs the
 * tensor-core kernel) and returns the same result bit for bit.  Its scratch and
 * tables live in fixed-size static device arrays that every GPU loading the
 * library holds until exit (about 10 MB).  Limits: b in {4, 8, 16} and at
 * most 65536 blocks (b = 4, 8) or 16384 blocks (b = 16) per call; larger
 * requests return AQMP_E_ARG.  The first call on a device looks up the
 * arrays' device addresses and should come before any stream capture.  A
 * call cannot be captured into a CUDA graph (it waits for `stream` and reads
 * a status word back): on a capturing stream it returns AQMP_E_UNSUPPORTED
 * and leaves the stream untouched.  Calls share the arrays and synchronise
 * `stream` before returning, on an error too once work was queued; GPU work
 * of two calls must not overlap (this function serialises its callers). */
int aqmp_correlate_noalloc(int b, int dict_id, const uint8_t *blocks, int64_t L, float *corr,
                           void *stream);

/* Check of the failure path (no counterpart in the paper): runs one thread
 * that waits, with the library's bounded device wait, on a barrier nothing
 * ever arrives on.  It must give up after `limit_ms` (1..5000) and report it:
 * the expected return is AQMP_E_TIMEOUT, after which the device stays usable.
 * AQMP_OK would mean the wait was not bounded. */
int aqmp_selftest_wait(int limit_ms, void *stream);

/* The rounding every exact correlation ends in: each of n integers T
 * (device memory, two int64 words per value, low word first, two's
 * complement, |T| < 2^112) becomes the double-float
 * (RN(T), RN(T - RN(T))) 2^-96, ties to even, written to `out` (device,
 * n float pairs; a zero low word carries the sign of T).  For tests of that
 * rounding against exact integer arithmetic.  Synchronises `stream`.  Errors: AQMP_E_ARG (NULL or
 * unaligned pointers, n out of [0, 2^31)), AQMP_E_CUDA. */
int aqmp_selftest_round(const int64_t *words, int64_t n, float *out, void *stream);

/* ---- Codec stages around the encoder (Section 2.3 and Appendix A) ----
 * Step (i) converts the channels of an image to RGB or YCbCr and codes each
 * channel on its own; step (iii) applies a lossless coder (DEFLATE) to the
 * MP output; the decoder reverses the three steps.  The paper fixes neither
 * the YCbCr variant nor the layout of the MP output; this library's choices:
 *  - YCbCr is the full-range JFIF matrix (ITU-T T.871) evaluated exactly in
 *    integers, each coefficient rounded to 16 fractional bits, rounding half
 *    up and clamping to [0, 255]; greys map to themselves.
 *  - The bitstream (the input of the lossless stage) lists, per plane, the
 *    leaves in canonical (depth-first) order.  A leaf's position is implied by
 *    that order and by the leaf sizes, as in the paper's decoder (set_block
 *    places blocks by the quadtree traversal order), so only sizes, step
 *    counts, atom indices and FP32 coefficients are stored.  Little-endian:
 *      "AQMP", u8 version = 1, u8 color, u8 dict_id, u8 0, u16 min_block,
 *      u16 max_block, u32 n_planes; per plane u32 h, w, n_leaves, n_atoms;
 *      then per plane: n_leaves u8 levels log2(max_block / b), n_leaves
 *      LEB128 step counts, n_atoms u16 atom indices, n_atoms f32 alpha.
 *  - DEFLATE itself is applied by the caller (the Python package uses zlib). */

#define AQMP_COLOR_PLANES 0       /* channels coded as given */
#define AQMP_COLOR_RGB    1       /* interleaved RGB, coded as R, G, B planes */
#define AQMP_COLOR_YCBCR  2       /* interleaved RGB, coded as Y, Cb, Cr planes */

/* Step (i) on the device: `img` is h x w x channels interleaved bytes with
 * `pitch` bytes per row; `planes` receives `channels` byte planes of h rows
 * of `plane_pitch` bytes, plane c starting at planes + c h plane_pitch.
 * AQMP_COLOR_YCBCR needs channels == 3 and converts RGB to Y, Cb, Cr; the
 * other modes copy the channels.  Both pointers are device memory; the
 * call enqueues on `stream` and returns.  Errors: AQMP_E_ARG. */
int aqmp_image_to_planes(const uint8_t *img, int h, int w, int channels, int64_t pitch, int color,
                         uint8_t *planes, int64_t plane_pitch, void *stream);

/* Decoder step (iii) on the device: `planes` holds `channels` decoded FP32
 * planes (as aqmp_decode writes them; plane c at planes + c h plane_pitch),
 * each value rounded to the nearest integer (ties to even) and clamped to
 * [0, 255]; AQMP_COLOR_YCBCR then converts Y, Cb, Cr to RGB.  `img`
 * receives h x w x channels interleaved bytes with `pitch` bytes per row.
 * Device memory; enqueues on `stream`.  Errors: AQMP_E_ARG. */
int aqmp_planes_to_image(const float *planes, int h, int w, int channels, int64_t plane_pitch, int color,
                         uint8_t *img, int64_t pitch, void *stream);

/* Size in bytes of the bitstream of `code` (host value). */
int aqmp_bitstream_size(const aqmp_code *code, uint64_t *bytes);

/* Writes the bitstream of `code` into the host buffer `buf` of `cap` bytes
 * (at least aqmp_bitstream_size); *len receives the bytes written; `color`
 * (AQMP_COLOR_*) is recorded for the decoder.  Errors: AQMP_E_ARG (NULL, or
 * cap too small), AQMP_E_UNSUPPORTED (a plane larger than 2^32 - 1 px). */
int aqmp_bitstream_write(const aqmp_code *code, int color, uint8_t *buf, uint64_t cap, uint64_t *len);

/* Header of a bitstream. */
typedef struct {
    int      version, color, dict_id, n_planes, min_block, max_block;
    uint64_t n_leaves, n_atoms;   /* totals over the planes */
} aqmp_bitstream_info;

/* Host-only parse of a bitstream: fills *info; when not NULL, `shapes`
 * (2 n_planes ints: h, w per plane), `leaves` (n_leaves) and `atoms`
 * (n_atoms) receive the planes' sizes and the leaves, in canonical order,
 * with their positions recovered from the traversal order (converged, flags
 * and the low coefficient words are not stored: zero).  Call once with NULL
 * arrays to learn the counts.  Errors: AQMP_E_ARG (malformed stream). */
int aqmp_bitstream_parse(const uint8_t *buf, uint64_t len, aqmp_bitstream_info *info, int *shapes,
                         aqmp_leaf *leaves, aqmp_atom *atoms);

/* A code object rebuilt from a bitstream (device arrays uploaded on the
 * current device), ready for aqmp_decode.  Errors: as aqmp_bitstream_parse,
 * AQMP_E_OOM, AQMP_E_CUDA. */
int aqmp_code_from_bitstream(const uint8_t *buf, uint64_t len, aqmp_code **out);

/* Number of atoms M of a dictionary at side b (2 b^2 or b^2), or < 0. */
int aqmp_num_atoms(int b, int dict_id);

/* Message of the calling thread's last failed call ("" if none). */
const char *aqmp_last_error(void);

/* Device time in milliseconds of the most recent aqmp_encode_planes,
 * aqmp_encode or aqmp_encode_batch call on the current device: CUDA events
 * recorded on the stream that runs the call's kernels, just before the first
 * of them (after the call's wait on the caller's stream) and just after the
 * last; host-side work of the call (argument checks, the read-back of the
 * counters) lies outside it.  *ms = -1 when no encode has completed on the
 * device.  Errors: AQMP_E_ARG (ms NULL), AQMP_E_CUDA. */
int aqmp_last_device_ms(double *ms);

/* Library version string. */
const char *aqmp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AQMP_H */
