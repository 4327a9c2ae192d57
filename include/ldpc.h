/*
 * ldpc.h -- C ABI of the GB300 (sm_103a) flooding Min-Sum LDPC decoder.
 *
 * The decoder implements Algorithm 1 of arXiv 2507.10424 ("A mapping of the Min-Sum
 * decoder to reduction operations, and its implementation using CUDA kernels"):
 *   - the parity matrix H is a run-time argument known only by its dimensions
 *     (Section I and the abstract);
 *   - check-node update, eq. (eta_update), computed through Observation 1 (the two
 *     smallest magnitudes and the first location of the smallest) and Observation 2
 *     (extrinsic sign = total sign product x own sign, sign(0) = +1, Section III);
 *   - variable-node update, eq. (lambda_j): s_j = r_j + sum over the checks of bit j,
 *     added in ascending check order starting from r_j;
 *   - hard decision, eq. (slice), and the syndrome test H b = 0 over GF(2), eq. (1)-(2),
 *     with per-frame early stop (the termination test of Algorithms 1 and 2).
 *
 * Conventions shared by every entry point:
 *   - LLRs are log P(bit=0)/P(bit=1): positive favours 0 and the hard decision is
 *     b_j = [s_j < 0]. The paper prints the opposite slicer ([s_j > 0] means 1), which
 *     is consistent with its sign-product rule only for codes whose rows all have even
 *     weight; it is available as LDPC_FLAG_PAPER_SLICER.
 *   - Buffers are frame-major: frame f, bit j at [f * N + j].
 *   - Decoding is asynchronous on the handle's stream (ldpc_set_stream); errors that the
 *     host can detect are returned at once, and nothing is enqueued when a call fails.
 *   - The caller owns every input and output buffer; the handle owns the device copy
 *     of H and the decoding workspace, and frees both in ldpc_destroy.
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 *
 * Fixed-point mode (LDPC_MODE_FIXED): LLRs are quantised as
 * q = clamp(round_half_even(4 * llr), -127, 127) (int8, step 0.25); lambda, eta and s are
 * kept in [-32767, 32767] (int16 storage, int32 arithmetic, lambda and s saturate).
 * FP32 mode computes in binary32 with round-to-nearest; its results are bit-identical to
 * a sequential binary32 evaluation in the order stated above.
 */
#ifndef LDPC_H
#define LDPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldpc ldpc_t; /* opaque handle */

/* Status codes. */
#define LDPC_OK 0
#define LDPC_ERR_INVALID_ARG (-1)  /* a size, flag or option is out of range */
#define LDPC_ERR_INVALID_H (-2)    /* H entry not 0/1, duplicate/out-of-range index, row of weight 1, E >= 2^31 */
#define LDPC_ERR_BAD_POINTER (-3)  /* NULL where required, or host memory where device memory is required */
#define LDPC_ERR_OOM (-4)          /* device or host allocation failed */
#define LDPC_ERR_CUDA (-5)         /* a CUDA runtime call failed; see ldpc_last_cuda_error */
#define LDPC_ERR_TIMEOUT (-6)      /* a bounded wait inside a kernel ran out (ldpc_check_device) */
#define LDPC_ERR_DEVICE_CHECK (-7) /* the debug checks (ldpc_set_debug) found a NaN LLR or an index out of range */
#define LDPC_ERR_UNSUPPORTED (-8)  /* the request needs a feature this build or device lacks */

/* Arithmetic modes. */
#define LDPC_MODE_FP32 0
#define LDPC_MODE_FIXED 1

/* H formats for ldpc_create_ex. */
#define LDPC_H_DENSE_U8 0   /* h_a: uint8 [M][N], row-major, entries 0/1; h_b unused */
#define LDPC_H_PACKED_U32 1 /* h_a: uint32 [M][ceil(N/32)]; bit (j%32) of word j/32 is H(i,j); unused high bits 0 */
#define LDPC_H_CSR 2        /* h_a: int64 row_ptr [M+1]; h_b: int32 col_idx [row_ptr[M]] (any order in a row) */

/* LLR element types for ldpc_decode_ex. */
#define LDPC_LLR_F32 0
#define LDPC_LLR_I8 1 /* already quantised (step 0.25); fixed mode only */

/* Flags for ldpc_create_ex. */
#define LDPC_FLAG_PAPER_SLICER 1 /* b_j = [s_j > 0], the slicer as printed in eq. (slice) */
#define LDPC_FLAG_DEBUG 2        /* device-side debug checks before every decode (ldpc_set_debug) */

/* Kernel variants (ldpc_set_variant). */
#define LDPC_VARIANT_AUTO 0     /* resident when a frame fits in shared memory, else streaming */
#define LDPC_VARIANT_STREAM 1   /* messages in HBM, frame-interleaved, two kernels per iteration */
#define LDPC_VARIANT_RESIDENT 2 /* one persistent kernel, frames resident in shared memory */
#define LDPC_VARIANT_DENSE 3    /* the paper's dense m x n map-reduce form (Algorithm 2): a
                                   baseline; FP32 only, at most 65535 frames per call, and
                                   4 M N bytes of workspace per frame */
#define LDPC_VARIANT_CLUSTER 4  /* one persistent kernel; a thread-block cluster of 2-16 CTAs
                                   keeps a tile of frames in its distributed shared memory,
                                   rows and columns split between the CTAs. For codes too
                                   large for one SM; slower than streaming there on GB300
                                   (scattered reads of other CTAs' shared memory), so it is
                                   never chosen by AUTO */

/*
 * ldpc_create: build a decoder for the M x N parity matrix H (host pointer, dense uint8,
 * row-major, entries 0 or 1), FP32 mode, on the current CUDA device.
 * Returns NULL on failure; ldpc_last_error() then gives the reason.
 * H ingestion (Section II-B, the sets N_i and M_j): the rows and columns of H become a
 * CSR/CSC edge list and bit-packed rows on the device; H is not retained by reference.
 * Rows of weight 0 are always satisfied; rows of weight 1 are rejected (their minimum
 * over the other neighbours is empty).
 */
ldpc_t *ldpc_create(int32_t M, int32_t N, const uint8_t *H);

/* ldpc_create_ex: as ldpc_create, with the H format (LDPC_H_*), mode (LDPC_MODE_*) and
 * flags (LDPC_FLAG_*) given. h_a / h_b are host pointers as described for each format. */
ldpc_t *ldpc_create_ex(int32_t M, int32_t N, int32_t h_format, const void *h_a, const void *h_b,
                       int32_t mode, int32_t flags);

/*
 * ldpc_decode: decode `frames` FP32 LLR frames (device pointer llr [frames][N]) with at
 * most max_iter flooding iterations and early stop (syndrome tested before the first
 * iteration and after every iteration). Writes the hard decisions (device uint8
 * out_bits [frames][N], values 0/1) and the iteration count per frame (device int32
 * out_iters [frames]: 0 if the input already satisfies H, else the iteration after which
 * the syndrome was zero, else max_iter). In fixed mode the LLRs are quantised first.
 * frames == 0 is a no-op; frames < 0 or max_iter < 0 give LDPC_ERR_INVALID_ARG, and so
 * does a streaming-variant call with more than 2,097,120 frames (split larger batches).
 */
int ldpc_decode(ldpc_t *h, const float *llr, int32_t frames, int32_t max_iter, uint8_t *out_bits,
                int32_t *out_iters);

/* ldpc_decode_i8: as ldpc_decode for pre-quantised int8 LLRs (device pointer, step 0.25);
 * fixed mode only (LDPC_ERR_INVALID_ARG otherwise). */
int ldpc_decode_i8(ldpc_t *h, const int8_t *llr_q, int32_t frames, int32_t max_iter,
                   uint8_t *out_bits, int32_t *out_iters);

/*
 * ldpc_decode_ex: the general form. llr_dtype is LDPC_LLR_F32 or LDPC_LLR_I8.
 * early_stop = 0 runs exactly max_iter iterations (out_iters = max_iter for every frame).
 * check_every >= 1: with early stop, the syndrome is tested before the first iteration
 * and after iterations that are multiples of check_every (the paper tests every 6th).
 * out_ok (nullable, device uint8 [frames]): 1 if the returned bits satisfy H.
 * out_soft (nullable, device float [frames][N]): the posterior s of the returned bits,
 * in LLR units (fixed mode: s / 4, exact).
 */
int ldpc_decode_ex(ldpc_t *h, const void *llr, int32_t llr_dtype, int32_t frames, int32_t max_iter,
                   int32_t early_stop, int32_t check_every, uint8_t *out_bits, int32_t *out_iters,
                   uint8_t *out_ok, float *out_soft);

/*
 * ldpc_decode_host: ldpc_decode_ex with HOST buffers (preferably pinned): the LLRs are
 * copied to the device in chunks, decoded and the results copied back, with the copies
 * of one chunk overlapping the decoding of another (two device staging slots, kept by
 * the handle and grown as needed). Chunks are about a quarter of the frames (at least
 * 1024, at most 512 MiB of LLRs); with enough frames their sizes ramp up from an eighth
 * of a chunk, doubling, and back down at the end, since nothing overlaps the first
 * chunk's input copy or the last chunk's output copy. Synchronous: returns when the
 * results are in the host buffers. out_ok and out_soft may be NULL. Errors: those of
 * ldpc_decode_ex, and LDPC_ERR_BAD_POINTER for a null llr_host, bits_host or iters_host.
 */
int ldpc_decode_host(ldpc_t *h, const void *llr_host, int32_t llr_dtype, int32_t frames,
                     int32_t max_iter, int32_t early_stop, int32_t check_every,
                     uint8_t *bits_host, int32_t *iters_host, uint8_t *ok_host, float *soft_host);

/*
 * ldpc_decode_noalloc: ldpc_decode_ex without any device allocation. The paper has no
 * counterpart; this is a service entry point of this library.
 *
 * For callers that cannot allocate device memory while they decode: a serving loop that
 * must not stall on the allocator (cudaMalloc/cudaFree may synchronise the device), a
 * process whose device memory is already held by another allocator, or an embedding
 * that forbids allocation after start-up. It runs the streaming kernels with their
 * scratch taken from one static device array of LDPC_NOALLOC_SCRATCH_BYTES (32 MiB).
 * The array is mapped on a device when the first handle is created there (ldpc_create /
 * ldpc_create_ex fail with LDPC_ERR_OOM if it cannot be) and stays until the process
 * exits; this entry point itself maps and allocates nothing. The kernels' code is loaded
 * by the CUDA runtime on first use (lazy module loading, its default): a caller that can
 * allocate nothing at all after start-up makes one decode in each mode it uses at
 * start-up, or runs with CUDA_MODULE_LOADING=EAGER.
 *
 * Arguments and results are those of ldpc_decode_ex (device pointers). The scratch a
 * call needs is Fp * (S * m + N * (m + r) + max_iter + 15) + 256 bytes, with Fp = frames
 * rounded up to a multiple of 256, m = 4 (FP32) or 2 (fixed), r = 4 or 1, and S message
 * slots per frame: 8 M when no row has more than 8 edges, 16 M when none has more than 16,
 * else E. A larger request returns LDPC_ERR_INVALID_ARG without launching anything. The
 * current device must be the handle's device (else LDPC_ERR_INVALID_ARG). The handle's
 * debug checks (ldpc_set_debug) do not run on this entry point.
 * Every call uses the same array and each clears what must start from zero; calls whose
 * work overlaps on the GPU (other streams, or other handles) race on it and must be
 * serialised by the caller. It does not set ldpc_last_error().
 */
#define LDPC_NOALLOC_SCRATCH_BYTES (32u << 20)
int ldpc_decode_noalloc(ldpc_t *h, const void *llr, int32_t llr_dtype, int32_t frames,
                        int32_t max_iter, int32_t early_stop, int32_t check_every,
                        uint8_t *out_bits, int32_t *out_iters, uint8_t *out_ok, float *out_soft);

/*
 * Learned normalised / offset Min-Sum (an extension of eq. eta_update; the paper has
 * plain Min-Sum only). Each extrinsic magnitude m of the check update becomes
 * max(fma(alpha, m, -beta), 0) in binary32, with (alpha, beta) chosen by the iteration t
 * and by the class of the edge's bit: classes are the distinct column weights of H in
 * ascending order (one class for a regular code). alpha = 1, beta = 0 is plain Min-Sum,
 * bit for bit.
 *
 * ldpc_classes: number of classes and (degrees, nullable) the column weight of each.
 */
int ldpc_classes(const ldpc_t *h, int32_t *n_classes, int32_t *degrees);

/* ldpc_set_weights: decode with learned weights from now on (FP32 mode; decodes in fixed
 * mode then return LDPC_ERR_UNSUPPORTED). alpha, beta: host [n_rows][n_classes]; iteration
 * t uses row min(t, n_rows) - 1. n_rows = 0 returns to plain Min-Sum. */
int ldpc_set_weights(ldpc_t *h, int32_t n_rows, const float *alpha, const float *beta);

/* ldpc_train_workspace_size: device bytes that ldpc_train_forward/backward need for
 * `frames` frames and `iters` unrolled iterations: about frames x (12 N + 8 E + iters x 12 M)
 * bytes when no row of H has more than 16 edges (each check keeps min0, min1 and one word
 * holding its minimum locations, sign parity and sign bits per iteration), plus frames x
 * iters x E bytes (a sign byte per edge) for codes with longer rows. */
int ldpc_train_workspace_size(ldpc_t *h, int32_t frames, int32_t iters, uint64_t *bytes);

/* ldpc_train_forward: `iters` flooding iterations (no early stop) of the learned decoder
 * on FP32 LLRs (device [frames][N]); alpha, beta: device [iters][n_classes]. Writes the
 * posteriors to device float `soft`: [frames][N] after the last iteration (soft_every = 0;
 * equal to ldpc_decode_ex's out_soft with the same weights and early_stop = 0), or
 * [iters][frames][N] after every iteration (soft_every = 1). Keeps, in `work` (device,
 * caller-owned), the per-iteration compressed check state the backward pass needs. */
int ldpc_train_forward(ldpc_t *h, const float *llr, int32_t frames, int32_t iters,
                       const float *alpha, const float *beta, float *soft, int32_t soft_every,
                       void *work, uint64_t work_bytes);

/* ldpc_train_backward: adjoint of the preceding ldpc_train_forward (same frames, iters,
 * weights, soft_every and work): from grad_soft (device, shaped like that call's `soft`:
 * the loss gradient w.r.t. the posteriors) computes grad_alpha and grad_beta (device
 * [iters][n_classes], overwritten). Messages are rebuilt per iteration from the saved
 * state; the gradient follows the edge attaining each minimum (a subgradient) and treats
 * signs as constant. */
int ldpc_train_backward(ldpc_t *h, int32_t frames, int32_t iters, const float *alpha,
                        const float *beta, const float *grad_soft, int32_t soft_every,
                        float *grad_alpha, float *grad_beta, void *work, uint64_t work_bytes);

/*
 * Batched decoding of several codes of uneven size in ONE persistent launch (FP32 mode).
 * The paper decodes one frame of one code at a time; this batches frames of many codes.
 * The batch refers to existing handles (which must outlive it; all on the current
 * device, all with or all without LDPC_FLAG_PAPER_SLICER, each small enough for the
 * resident variant's sliced layout). Its kernel takes (code, frame) tiles from one work
 * counter, largest codes first; a code whose frame fits in shared memory keeps its
 * messages there. A larger code is by default decoded by the streaming kernels on one of
 * two streams forked from (and joined back to) the batch's stream (the large codes
 * alternate between them), alongside the persistent kernel; ldpc_batch_set_large_codes(b, 0) puts it in the persistent launch
 * instead, with a per-CTA slot of the batch's global scratch. Either way the launch is
 * one recordable unit. Results equal ldpc_decode_ex with check_every = 1 on each code.
 *
 * ldpc_batch_create: NULL on failure (bad handle, mixed slicers, device mismatch, OOM).
 */
typedef struct ldpc_batch ldpc_batch_t;
ldpc_batch_t *ldpc_batch_create(int32_t n_codes, ldpc_t *const *codes);

/* ldpc_batch_set_stream: stream of the batch's launches (a non-default stream is needed
 * for ldpc_batch_capture). */
int ldpc_batch_set_stream(ldpc_batch_t *b, void *cuda_stream);

/* ldpc_batch_set_io: device buffers of code `code` for the next prepare: llr [frames][N],
 * out_bits [frames][N], out_iters [frames], out_ok / out_soft nullable. frames may be 0. */
int ldpc_batch_set_io(ldpc_batch_t *b, int32_t code, const float *llr, int32_t frames,
                      uint8_t *out_bits, int32_t *out_iters, uint8_t *out_ok, float *out_soft);

/* ldpc_batch_prepare: upload the per-code descriptors and the tile list for max_iter and
 * early_stop (synchronous; waits for the batch's stream). */
int ldpc_batch_prepare(ldpc_batch_t *b, int32_t max_iter, int32_t early_stop);

/* ldpc_batch_launch: enqueue the prepared decode (a counter reset and the persistent
 * kernel, plus the streaming kernels of the large codes between a fork and a join). */
int ldpc_batch_launch(ldpc_batch_t *b);

/* ldpc_batch_set_large_codes: codes too large for shared memory are decoded by the
 * streaming kernels (streaming = 1, the default) or inside the persistent launch from
 * global scratch (0). Takes effect at the next ldpc_batch_prepare. LDPC_ERR_INVALID_ARG
 * for other values. */
int ldpc_batch_set_large_codes(ldpc_batch_t *b, int32_t streaming);

/* ldpc_batch_set_sm_split: with large codes decoded by the streaming kernels beside the
 * persistent launch, run the persistent kernel on at most `sms` SMs (its CTAs) and size
 * the streaming kernels' persistent check passes to the other SMs, so that the resident
 * tiles (bound by shared memory and instruction issue) and the streaming passes (bound by
 * DRAM bandwidth) run side by side on disjoint SMs instead of taking turns on all of them.
 * 0 (default): no split. Results do not depend on it. Takes effect at the next
 * ldpc_batch_prepare; ldpc_batch_autotune tries several splits. LDPC_ERR_INVALID_ARG for
 * sms < 0 or sms >= the device's SM count. ldpc_batch_get_sm_split reads it back. */
int ldpc_batch_set_sm_split(ldpc_batch_t *b, int32_t sms);
int ldpc_batch_get_sm_split(const ldpc_batch_t *b, int32_t *sms);

/* ldpc_batch_decode: ldpc_batch_prepare then ldpc_batch_launch. */
int ldpc_batch_decode(ldpc_batch_t *b, int32_t max_iter, int32_t early_stop);

/* ldpc_batch_capture: record the prepared launch in a CUDA graph (on the batch's stream);
 * ldpc_batch_replay launches that graph. Prepare and capture again after changing the
 * buffers, the iteration limit or the CTA size. */
int ldpc_batch_capture(ldpc_batch_t *b);
int ldpc_batch_replay(ldpc_batch_t *b);

/* ldpc_batch_set_threads: CTA size of the batch kernel (64..1024, a multiple of 32).
 * ldpc_batch_set_tile_frames: at most 1, 2 or 4 frames interleaved per tile for the codes
 * kept in shared memory (default 4; a code whose frames do not fit that many uses fewer);
 * takes effect at the next ldpc_batch_prepare. ldpc_batch_get_tile_frames reads it back.
 * ldpc_batch_autotune: times the decode prepared for max_iter / early_stop on the buffers
 * set with ldpc_batch_set_io, for every cap on the frames per tile x CTA size, keeps the
 * fastest pair, then (with streamed large codes) times SM splits (ldpc_batch_set_sm_split)
 * and leaves the batch prepared with the fastest; best_threads and best_ms
 * (nullable) receive the CTA size and the time of one decode; on an error the cap and CTA
 * size the batch had stay in force (prepare it again before launching). With early stop a
 * tile runs until its last frame stops, so narrower tiles can win. */
int ldpc_batch_set_threads(ldpc_batch_t *b, int32_t threads);
int ldpc_batch_set_tile_frames(ldpc_batch_t *b, int32_t max_frames_per_tile);
int ldpc_batch_get_tile_frames(const ldpc_batch_t *b, int32_t *max_frames_per_tile);
int ldpc_batch_autotune(ldpc_batch_t *b, int32_t max_iter, int32_t early_stop,
                        int32_t *best_threads, float *best_ms);

/* ldpc_batch_info: codes, prepared tiles, CTA size, codes kept in shared memory. */
int ldpc_batch_info(const ldpc_batch_t *b, int32_t *n_codes, int32_t *n_tiles, int32_t *threads,
                    int32_t *codes_in_shared_memory);

/* ldpc_batch_destroy: waits for the batch's stream, frees it (not the handles). */
void ldpc_batch_destroy(ldpc_batch_t *b);

/* ldpc_set_stream: decode on this cudaStream_t (NULL = legacy default stream). */
int ldpc_set_stream(ldpc_t *h, void *cuda_stream);

/* ldpc_set_mode: switch between LDPC_MODE_FP32 and LDPC_MODE_FIXED. */
int ldpc_set_mode(ldpc_t *h, int32_t mode);

/* ldpc_set_variant: choose the kernel variant (LDPC_VARIANT_*). RESIDENT fails with
 * LDPC_ERR_UNSUPPORTED when one frame of this code does not fit in shared memory, CLUSTER
 * when one frame does not fit the shared memory of the requested (or any) cluster. */
int ldpc_set_variant(ldpc_t *h, int32_t variant);

/*
 * ldpc_set_tuning: launch shape of the resident kernel (0 = automatic for each field).
 * frames_per_tile in {0, 1, 2, 4}: frames interleaved per CTA tile; threads: CTA size
 * (a multiple of 32, at most 1024); index_placement: 1 = the code's index arrays are copied
 * to shared memory, 2 = read from global memory (leaves room for more CTAs per SM).
 * Results do not depend on the tuning.
 * LDPC_ERR_UNSUPPORTED when the requested shape does not fit this code (the previous
 * tuning stays in force), LDPC_ERR_INVALID_ARG for values outside these sets. (The paper
 * tunes blocks and threads per kernel by hand, Section IV; this is the knob the
 * autotuner turns.)
 */
int ldpc_set_tuning(ldpc_t *h, int32_t frames_per_tile, int32_t threads, int32_t index_placement);

/*
 * ldpc_autotune: time launch shapes on this device for this code and mode, and keep the
 * fastest.
 *   - When the next decode runs the resident kernel: its frames per tile x index
 *     placement x CTA size, on min(frames, 16384) frames (as ldpc_set_tuning would set).
 *   - When it runs the streaming kernels: the staged check pass's warps per CTA x
 *     stages, and the unstaged kernel, on min(frames, 2048) frames (as
 *     ldpc_set_stream_staging would set).
 * The timing uses max_iter iterations without early stop. Allocates and frees its own
 * temporary device buffers; synchronises the handle's stream. best_ms (nullable) receives
 * the time of one decode of that many frames with the chosen shape.
 * LDPC_ERR_UNSUPPORTED when the code has no resident plan (resident), or no padded row
 * layout, i.e. rows longer than 16 edges (streaming).
 */
int ldpc_autotune(ldpc_t *h, int32_t frames, int32_t max_iter, float *best_ms);

/*
 * ldpc_autotune_data: as ldpc_autotune, but each shape decodes the caller's frames with the
 * caller's early-stop settings, so the choice fits workloads whose frames stop at
 * different iterations (a tile of several frames runs until its last frame stops, which
 * favours narrower tiles than timing without early stop does).
 *   llr         device pointer, FP32 [frames][N], frame-major (as ldpc_decode_ex with
 *               LDPC_LLR_F32); only the first min(frames, 65536) (resident) or
 *               min(frames, 2048) (streaming) frames are decoded; read only.
 *   early_stop  0 or 1; check_every >= 1 (as ldpc_decode_ex).
 * Errors: LDPC_ERR_BAD_POINTER for a null handle or an llr that is not device memory,
 * LDPC_ERR_INVALID_ARG for frames <= 0, max_iter < 0, check_every < 1 or early_stop not 0/1,
 * and the errors of ldpc_autotune.
 */
int ldpc_autotune_data(ldpc_t *h, const float *llr, int32_t frames, int32_t max_iter,
                       int32_t early_stop, int32_t check_every, float *best_ms);

/*
 * ldpc_set_debug: device-side debug checks on (1) or off (0). While on, ldpc_decode,
 * ldpc_decode_i8, ldpc_decode_ex and ldpc_decode_host first run checking kernels on the
 * handle's stream over every index array the decode kernels read through (CSR/CSC
 * offsets and indices, the sliced and padded layouts' slot ids, column positions, slice
 * degrees and weight classes: each within the array it indexes) and over the caller's FP32
 * LLRs (no NaN: the decoder does not define it), then synchronise the stream and read the
 * result. A violation returns LDPC_ERR_DEVICE_CHECK and no decode kernel is launched; the
 * outputs are left untouched. Slow (a stream synchronisation per call): for testing and
 * diagnosis. Also switched on at create by LDPC_FLAG_DEBUG, or by the environment variable
 * LDPC_DEBUG=1 (read by ldpc_create / ldpc_create_ex). Errors: LDPC_ERR_INVALID_ARG for
 * on not 0/1; LDPC_ERR_OOM if the report buffer cannot be allocated.
 *
 * ldpc_debug_report: the first violation of the last decode that the checks refused, then
 * clears it. what: 0 none, 1 a NaN LLR (where = frame * N + bit), 2 an index array (where
 * = array id << 40 | entry; ids: 1 row offsets, 2 column offsets, 3 column index of an
 * edge, 4 edge of a CSC entry, 5 column class, 6 row slice offsets, 7 column slice
 * offsets, 8 row slice degree, 9 column slice degree, 10 column position of a row slot,
 * 11 row slot of a column entry, 12 column position of a bit, 13 class of a row slot,
 * 14 column of a padded row slot, 15 padded row degree, 16 padded slot of an edge, 17 class
 * of a padded row slot). what and where are host pointers.
 */
int ldpc_set_debug(ldpc_t *h, int32_t on);
int ldpc_debug_report(ldpc_t *h, int32_t *what, int64_t *where);

/* ldpc_get_tuning: the resident launch shape in force for the current mode. */
int ldpc_get_tuning(const ldpc_t *h, int32_t *frames_per_tile, int32_t *threads,
                    int32_t *index_placement);

/* ldpc_set_stream_group: frame grouping of the streaming variant. The batch is decoded in
 * groups of frames, one group after another, each through all its iterations, so that a
 * group's messages can stay in L2. -1 (default): no groups; 0: groups sized so that a
 * group's working set (about frames x (E m + N (m + r)) bytes) fits half the L2 cache, when
 * the whole batch does not; > 0 (a multiple of 32): groups of this many frames. Results do
 * not depend on the grouping; small groups leave the GPU partly idle, which is why it is
 * off by default. Returns LDPC_ERR_INVALID_ARG for other values. */
int ldpc_set_stream_group(ldpc_t *h, int32_t frames_per_group);

/*
 * ldpc_set_stream_staging: shape of the streaming variant's check pass for codes whose
 * rows have at most 16 edges. Row i then owns 8 or 16 message slots (a padded row
 * layout). Each warp of a persistent kernel keeps `stages` shared-memory stages in
 * flight. Into each stage, the TMA engine's bulk asynchronous copies (cp.async.bulk)
 * bring one row's gathered posteriors s_j and old messages for 32 x frames_per_lane
 * frames, completing on an mbarrier, while the warp computes an earlier row (Section
 * III's row reductions).
 *   warps_per_cta in {0 (automatic: 12; for FP32 codes with compressed messages on rows
 *                     of 16 slots, the largest of 12, 8 and 4 whose stages fit the
 *                     device's shared memory), 1..12};
 *   stages in {-1 (off: one thread per row and frame vector loads its row itself),
 *              0 (automatic: 2), 2..8};
 *   frames_per_lane in {0 (automatic: the mode's 16-byte vector, 4 FP32 or 8 int16 frames),
 *                       1, 2, 4, 8 (at most the automatic width)}.
 * Results do not depend on the shape. A shape whose shared memory does not fit the device
 * falls back to the unstaged kernel. LDPC_ERR_INVALID_ARG for other values.
 */
int ldpc_set_stream_staging(ldpc_t *h, int32_t warps_per_cta, int32_t stages, int32_t frames_per_lane);

/*
 * ldpc_set_stream_messages: how the streaming variant keeps the check-to-bit messages of
 * FP32 codes whose rows have at most 16 edges. compressed = 1 (default): per row and frame
 * only the two smallest magnitudes min0 <= min1 of Observation 1, the first location of
 * min0 and the signs of Observation 2 (12 bytes per row; every message eta_ij of eq.
 * (eta_update) is rebuilt from them exactly), so the per-edge messages never travel
 * through DRAM; it needs the staged check pass (ldpc_set_stream_staging with stages >= 2).
 * compressed = 0: one stored message per edge slot. Results do not depend on the choice.
 * Fixed-point mode and rows longer than 16 edges always keep per-edge messages.
 * ldpc_autotune also chooses this for FP32 codes. LDPC_ERR_INVALID_ARG for other values.
 * ldpc_get_stream_messages: 1 when the next streaming decode keeps compressed messages.
 */
int ldpc_set_stream_messages(ldpc_t *h, int32_t compressed);
int ldpc_get_stream_messages(const ldpc_t *h, int32_t *compressed);

/* ldpc_get_stream_staging: the staging in force (stages 0 when off; frames_per_lane 0 when
 * automatic). */
int ldpc_get_stream_staging(const ldpc_t *h, int32_t *warps_per_cta, int32_t *stages,
                            int32_t *frames_per_lane);

/*
 * ldpc_read_messages: the check-to-bit messages eta_ij of eq. (eta_update) after the last
 * iteration of the handle's last decode, for tests and diagnosis. They are available when
 * that decode (ldpc_decode_ex or a function built on it) ran the streaming variant without
 * early stop and without frame groups, since its messages then remain in the handle's
 * workspace; the resident, cluster and dense variants keep them on chip and discard them.
 *   frames  how many frames to read (the first ones of that decode), 0 .. its frame count;
 *   out     device float [frames][E], frame-major; edge e in CSR order (rows ascending, the
 *           columns of a row ascending); values in LLR units (fixed mode: eta / 4, exact).
 * Asynchronous on the handle's stream. Errors: LDPC_ERR_UNSUPPORTED when the last decode
 * left no messages, LDPC_ERR_INVALID_ARG for frames < 0 or more frames than it decoded,
 * LDPC_ERR_BAD_POINTER for a null handle or an out that is not device memory. frames = 0 is
 * a no-op.
 */
int ldpc_read_messages(ldpc_t *h, int32_t frames, float *out);

/*
 * ldpc_check_device: waits for the handle's stream, then reads and clears the handle's
 * device error word. That word covers this handle's decodes, including a batch's large
 * codes, which run the streaming kernels on their code's handle. Returns LDPC_OK, or
 * LDPC_ERR_TIMEOUT when a bounded wait inside a kernel ran out since the last check. The
 * kernel then gave up its waits, let its own copies in flight land, and returned, so the
 * outputs of that decode are not valid. LDPC_ERR_CUDA when the stream reports an error.
 */
int ldpc_check_device(ldpc_t *h);

/*
 * ldpc_set_wait_limit: tries of each bounded wait in the staged kernels. One try waits at
 * most about 20 microseconds. The default 65536 bounds a wait near 1.3 s, far above any
 * real copy. A limit of 0 makes every wait give up at once, which is how the tests check
 * the timeout path without a fault. tries must be >= 0, else LDPC_ERR_INVALID_ARG.
 */
int ldpc_set_wait_limit(ldpc_t *h, int32_t tries);

/*
 * ldpc_set_cluster_shape: launch shape of the cluster variant (0 = automatic for each field).
 * cluster_size in {0, 1, 2, 4, 8, 16}: CTAs per cluster (automatic: the smallest of 2, 4,
 * 8, 16 that holds a frame; 16 needs the device's non-portable cluster size);
 * frames_per_tile in {0, 1, 2, 4}: frames interleaved per tile (automatic: the most that
 * fit); threads in {0} or multiples of 32 in [64, 1024] (automatic: 1024). The CTAs of a
 * cluster split the rows and the columns of H by edge count; each needs 16-bit slot ids
 * (at most 65536 row slots and 65535 columns). Results do not depend on the shape.
 * LDPC_ERR_INVALID_ARG for values outside these sets; a shape that does not fit the code
 * shows up as LDPC_ERR_UNSUPPORTED from the cluster variant.
 */
int ldpc_set_cluster_shape(ldpc_t *h, int32_t cluster_size, int32_t frames_per_tile,
                           int32_t threads);

/* ldpc_get_cluster_shape: the cluster variant's shape in the current mode, and how many
 * clusters the device holds at once (any pointer may be NULL). LDPC_ERR_UNSUPPORTED when
 * no cluster shape fits. */
int ldpc_get_cluster_shape(const ldpc_t *h, int32_t *cluster_size, int32_t *frames_per_tile,
                           int32_t *threads, int32_t *clusters);

/* ldpc_get_variant: the variant the next decode will run (AUTO resolved). */
int ldpc_get_variant(const ldpc_t *h, int32_t *variant);

/* ldpc_reserve: pre-size the workspace for up to max_frames frames per call (otherwise
 * it grows on demand). Allocation happens here, never inside a timed decode. */
int ldpc_reserve(ldpc_t *h, int32_t max_frames);

/* ldpc_info: dimensions and degree statistics of H (any pointer may be NULL). */
int ldpc_info(const ldpc_t *h, int32_t *M, int32_t *N, int64_t *E, int32_t *max_dc,
              int32_t *max_dv);

/* ldpc_last_kernel_count: number of kernels the last decode call launched. */
int ldpc_last_kernel_count(const ldpc_t *h, int32_t *count);

/* ldpc_last_error: status of the last failing call on this host thread (0 if none). */
int ldpc_last_error(void);

/* ldpc_last_cuda_error: the cudaError_t behind the last LDPC_ERR_CUDA on this thread. */
int ldpc_last_cuda_error(void);

/* ldpc_strerror: static text for a status code. */
const char *ldpc_strerror(int status);

/* ldpc_destroy: free the handle (waits for its stream). NULL is ignored. */
void ldpc_destroy(ldpc_t *h);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_H */
