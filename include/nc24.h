/*
 * nc24 - per-token CDF step of a neural lossless text compressor, as a C ABI.
 *
 * The compressor follows arXiv 2602.19626 ("Nacrith"), Algorithm 1: for each
 * token a decoder-only transformer predicts the next-token distribution
 * (Sec. 3.2, Eq. lm), an adaptive log-space bias corrects it (Sec. 3.6), it is
 * mixed linearly with an online token N-gram (Sec. 3.4, Sec. 3.5), quantised
 * to an integer CDF totalling 2^24 with a floor per symbol (Sec. 3.3), and
 * coded by a 32-bit arithmetic coder (Sec. 3.8) that runs on the host.
 *
 * Conventions for every entry point:
 *  - Every call returns nc_status; no exception or signal crosses the ABI.
 *  - The caller owns every buffer it passes; the library never frees or keeps
 *    caller memory beyond the call.  The library owns all device state of a
 *    context and releases it in nc_ctx_destroy.
 *  - "host" pointers are ordinary (pageable or pinned) CPU memory; "device"
 *    pointers are CUDA global memory on the context's device.  Entry points
 *    that accept either say so and detect the kind with cudaPointerGetAttributes.
 *  - A context is not thread-safe; use one context per host thread.
 *  - After NC_ECUDA or NC_ETIMEOUT the context is poisoned: every later call
 *    except nc_ctx_destroy / nc_last_error returns NC_ESTATE.
 *  - Work is ordered on the context's CUDA stream (nc_config.cuda_stream, or
 *    a stream the library creates when it is NULL); calls that return host
 *    data synchronise that stream before returning.
 */
#ifndef NC24_H
#define NC24_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nc_ctx nc_ctx;

typedef enum {
  NC_OK = 0,
  NC_EINVAL = 1,    /* bad argument (null pointer, size out of range, unknown stream) */
  NC_ENOMEM = 2,    /* device or host allocation failed */
  NC_ECUDA = 3,     /* a CUDA call failed; context poisoned */
  NC_ETIMEOUT = 4,  /* a bounded device wait gave up; context poisoned */
  NC_ECORRUPT = 5,  /* container bytes are malformed or do not match the context */
  NC_ESTATE = 6,    /* call out of order (e.g. step twice without update) or poisoned ctx */
  NC_ENUMERIC = 7   /* non-finite probabilities, or the CDF residual underflows a floor */
} nc_status;

/* Weight storage formats.  Weights are always handed in as FP32 and
 * converted on the device: BF16 by round-to-nearest-even; FP8 E4M3 with one
 * FP32 scale per output channel, scale = amax/448, q = e4m3_rn(w/scale). */
enum { NC_FP32 = 0, NC_BF16 = 1, NC_FP8E4M3 = 2 };

/* Update rule after each coded token.
 *  NC_RULE_PAPER:     b -= alpha (p_tilde - e_t*)  (Sec. 3.6) and exponential
 *                     weights on the mixer, log w_j += eta log p_j(t*) (Sec. 3.5).
 *  NC_RULE_MIXED_NLL: one SGD step (rate alpha) of -log p_mix(t*) with respect
 *                     to b and the mixer log-weights. */
enum { NC_RULE_PAPER = 0, NC_RULE_MIXED_NLL = 1 };

/* Numeric path of the dense projections.  Encoder and decoder must use the
 * same path; the container records it.
 *  NC_PATH_GEMV: CUDA-core weight streaming, FP32 activations.
 *  NC_PATH_TC:   tcgen05 tensor-core GEMMs over the batch of streams, BF16
 *                activations (FP8 activations for NC_FP8E4M3), FP32 accumulation. */
enum { NC_PATH_GEMV = 0, NC_PATH_TC = 1 };

/* Host entropy coder of the coded streams.
 *  NC_CODER_ARITH: the 32-bit arithmetic coder (Sec. 3.8).
 *  NC_CODER_RANS:  rANS with a 64-bit state and 32-bit words, the ANS coder
 *                  named as future work (Sec. 6); same CDFs, same model
 *                  work, recorded in the container's flags (bit 4). */
enum { NC_CODER_ARITH = 0, NC_CODER_RANS = 1 };

typedef struct {
  /* model shape (Sec. 3.2): 30, 576, 9, 3, 1536, 49152 for SmolLM2-135M */
  int n_layers, d_model, n_heads, n_kv_heads, d_ffn, vocab;
  float rope_theta, rms_eps;        /* 1e5, 1e-5 */
  int ctx_len, slide;               /* KV window L and drop count C (Sec. 3.9): 2048, 512 */
  int ngram_order;                  /* 0..3; 0 disables the N-gram and the mix (Sec. 3.4) */
  int use_head;                     /* 1 enables the adaptive bias head (Sec. 3.6) */
  int cdf_log2_total;               /* log2 T, 24 (Sec. 3.3); 16..24 */
  uint32_t floor;                   /* per-symbol minimum count, 1 */
  float bias_lr;                    /* alpha, 1e-3 (Sec. 3.6) */
  float mix_eta;                    /* eta of the exponential weights, 1 (Sec. 3.5) */
  float w_llm_init;                 /* 0.85 (Sec. 3.5) */
  float temperature;                /* tau, 1.0 (Sec. 3.2) */
  int warmup;                       /* tokens coded with the LLM alone, 100 (Sec. 3.5) */
  int weight_fmt;                   /* NC_FP32 | NC_BF16 | NC_FP8E4M3 */
  int update_rule;                  /* NC_RULE_PAPER | NC_RULE_MIXED_NLL */
  int path;                         /* NC_PATH_GEMV | NC_PATH_TC */
  int max_streams;                  /* stream slots; also the largest batch of one step */
  int device;                       /* CUDA device ordinal */
  void* cuda_stream;                /* cudaStream_t to order work on, or NULL */
  int prefill_rows;                 /* encoder only: run the model over up to this many
                                       (stream, position) rows per forward pass, positions
                                       p .. p + m - 1 of every stream between window slides,
                                       with the per-token vocabulary pass and updates after
                                       it in order.  0 or 1: one position per step.  Changes
                                       no result; the decoder replays the same CDFs one
                                       position at a time.  At most 32768; two chunks are
                                       in flight (one forward beside the previous chunk's
                                       vocabulary passes), so it needs 2 x prefill_rows x
                                       (vocab x 4 + 1,584) bytes on the device for the
                                       logits and the N-gram states. */
  int skip;                         /* 1: confidence-based LLM skip (Sec. 3.7): a token whose
                                       N-gram distribution has entropy below 1.5 bits is
                                       coded with p = p_ng, and only the N-gram learns from
                                       it.  Needs ngram_order > 0.  Recorded in the
                                       container's flags. */
  int coder;                        /* NC_CODER_ARITH | NC_CODER_RANS */
} nc_config;

/* Fill *cfg with the SmolLM2-135M shape and the paper's defaults
 * (BF16 weights, paper rule, GEMV path, 1 stream, device 0). */
void nc_config_default(nc_config* cfg);

/* Create a context.  `weights` is a HOST buffer of nbytes = 4 * n_params FP32
 * values in this order: embedding [V, d]; per layer attn_norm [d],
 * wq [Hq*64, d], wk [Hkv*64, d], wv [Hkv*64, d], wo [d, Hq*64], ffn_norm [d],
 * w_gate [F, d], w_up [F, d], w_down [d, F]; final_norm [d].  Matrices are
 * [out, in] row-major; the LM head is tied to the embedding (Eq. lm without
 * an output bias).  The library copies and converts the weights; the caller
 * may free them on return.  Requires d_model and d_ffn multiples of 16,
 * d_model / n_heads == 64, n_heads a multiple of n_kv_heads, vocab < 65536,
 * ctx_len a power of two > slide > 0.  Errors: NC_EINVAL, NC_ENOMEM, NC_ECUDA. */
int nc_ctx_create(const nc_config* cfg, const void* weights, size_t nbytes, nc_ctx** out);

/* Release every device and host resource of the context (NULL is a no-op). */
void nc_ctx_destroy(nc_ctx* ctx);

/* Start a stream in a free slot with fresh state (empty KV window, b = 0,
 * w = (w_llm_init, 1 - w_llm_init), empty N-gram).  expected_len bounds the
 * number of tokens the stream will code (it sizes the N-gram tables, Sec. 3.4);
 * coding more returns NC_ESTATE.  stream_id is any non-negative caller key.
 * Errors: NC_EINVAL (id in use, no free slot, expected_len < 1), NC_ENOMEM. */
int nc_stream_open(nc_ctx* ctx, int32_t stream_id, int64_t expected_len);

/* Free a stream's slot and its N-gram tables.  Errors: NC_EINVAL (unknown id). */
int nc_stream_close(nc_ctx* ctx, int32_t stream_id);

/* One model step for n open streams (Algorithm 1, the body of the loop up to
 * probs_to_cdf): feeds each stream's previous token (BOS id 0 first), runs the
 * transformer with its KV window, the biased softmax, the N-gram and the mix,
 * and quantises to the integer CDF.
 *   stream_ids  HOST int32[n], distinct open streams.
 *   prev_tokens HOST int32[n] or NULL: the token each stream feeds; must equal
 *               the stream's last observed token (-1 for a fresh stream), it is
 *               a consistency check only.
 *   cdf_out     HOST or DEVICE uint32[n * (V + 1)] or NULL: row j receives
 *               stream j's CDF, cdf[0] = 0, cdf[V] = 2^cdf_log2_total.  NULL
 *               keeps the CDFs on the device for nc_update_bias.
 * Each stream must then be given its observed token by nc_update_bias before
 * its next step (else NC_ESTATE).  Errors: NC_EINVAL, NC_ESTATE, NC_ENUMERIC,
 * NC_ECUDA. */
int nc_step_cdf(nc_ctx* ctx, int n, const int32_t* stream_ids, const int32_t* prev_tokens,
                uint32_t* cdf_out);

/* Apply the updates after coding (Algorithm 1, "Update: N-gram, Mixer,
 * AdaptiveHead with t_i"): bias head and mixer by the configured rule, then
 * the N-gram counts, for n streams that have just stepped.
 *   stream_ids HOST int32[n]; observed HOST int32[n], tokens in [0, V).
 * Errors: NC_EINVAL, NC_ESTATE, NC_ECUDA. */
int nc_update_bias(nc_ctx* ctx, int n, const int32_t* stream_ids, const int32_t* observed);

/* Whole-stream compression into an NC05-style container (Sec. 3.12):
 * 9-byte header (magic "NC05", flags: bit 0 N-gram, 1 head, 2 skip,
 * 3 mixed-NLL rule, 4 rANS coder; tau as binary16, stream count), one
 * extension byte (weight format | path << 4), 12 bytes per stream (token
 * count, bit count, byte count, little-endian uint32), then the coded streams.
 *   tokens HOST array of n_streams HOST int32 pointers; lens HOST int64[n_streams].
 *   out    HOST buffer or NULL; *inout_nbytes holds its capacity on entry and
 *          the container size on return.  out == NULL only queries an upper
 *          bound of the size (no coding).
 * Streams are coded in one batch (at most max_streams), each in a fresh slot
 * that is closed again before return.  Errors: NC_EINVAL (too many streams,
 * buffer too small: *inout_nbytes then holds the size needed), NC_ENOMEM,
 * NC_ENUMERIC, NC_ECUDA. */
int nc_encode(nc_ctx* ctx, int n_streams, const int32_t* const* tokens, const int64_t* lens,
              uint8_t* out, size_t* inout_nbytes);

/* Per-kernel trace of one nc_encode_intervals call: for each kernel kind,
 * the launches, their summed device time (CUDA events around each launch on
 * the context's stream), the algorithmic bytes they move (weights, distinct
 * KV entries, activations and per-symbol vectors each read or written once)
 * and their arithmetic (2 per multiply-add of the projections and of the
 * attention's scores and weighted values). */
#define NC_TRACE_KINDS 16
typedef struct {
  int n_kinds;
  int graphed;                      /* 1: the traced steps were replayed from a CUDA graph */
  char name[NC_TRACE_KINDS][32];
  int64_t launches[NC_TRACE_KINDS];
  double ms[NC_TRACE_KINDS];
  double bytes[NC_TRACE_KINDS];
  double flops[NC_TRACE_KINDS];
} nc_trace;

/* The device half of nc_encode: per-token CDF steps for n_streams streams
 * whose tokens are already on the device, producing each token's coder
 * interval instead of the bitstream.
 *   tokens_dev    DEVICE int32, stream j's tokens at tokens_dev + offsets[j].
 *   offsets, lens HOST int64[n_streams].
 *   intervals_dev DEVICE uint32[n_streams][stride][2]: (cdf[t_i], cdf[t_i + 1])
 *                 of token i of stream j (Algorithm 1, probs_to_cdf then the
 *                 interval handed to ArithEncoder.encode); stride >= max lens.
 *   trace         NULL, or a HOST nc_trace filled per kernel kind; tracing
 *                 launches every kernel eagerly between CUDA events (slower).
 * Streams occupy fresh slots that are released before return.  Without a
 * trace the steps are replayed from a captured CUDA graph, asynchronously on
 * the context's stream; the call returns after the last step is enqueued
 * and the status words were read (one synchronisation at the end).
 * Errors: NC_EINVAL, NC_ENOMEM, NC_ENUMERIC, NC_ESTATE, NC_ECUDA. */
int nc_encode_intervals(nc_ctx* ctx, int n_streams, const int32_t* tokens_dev,
                        const int64_t* offsets, const int64_t* lens, uint32_t* intervals_dev,
                        int64_t stride, nc_trace* trace);

/* nc_encode_intervals that also returns the intermediate distributions of
 * one token of every stream, as the encoder computed them (the prefill
 * forward when prefill_rows > 1, else the per-token step): at token index
 * probe_pos (0-based) of each stream with more than probe_pos tokens, row j
 * of z (the logits, Eq. lm), p_tilde (the biased LLM distribution, Sec. 3.6),
 * p_ng (the N-gram distribution, Sec. 3.4) and p (the binary32 probabilities
 * handed to the quantiser) receives stream j's values.  z, p_tilde, p_ng, p:
 * DEVICE float[n_streams * V] each, any may be NULL; rows of streams that
 * are too short are left as they were.  Synchronous like nc_encode_intervals
 * without a trace.  Errors: those of nc_encode_intervals, and NC_EINVAL for
 * probe_pos < 0 or a probe buffer that is not device memory. */
int nc_encode_probe(nc_ctx* ctx, int n_streams, const int32_t* tokens_dev, const int64_t* offsets,
                    const int64_t* lens, uint32_t* intervals_dev, int64_t stride, int64_t probe_pos, float* z,
                    float* p_tilde, float* p_ng, float* p);

/* Mirror of nc_encode.  tokens_out: HOST array of HOST int32 pointers, one
 * per stream, each with room for that stream's token count; lens_out HOST
 * int64[stream count].  A NULL tokens_out only reads the header: lens_out
 * then receives the token counts (query).  Errors: NC_ECORRUPT (bad magic,
 * truncated or inconsistent table, flags / tau / path differ from the
 * context), NC_EINVAL, NC_ENOMEM, NC_ECUDA. */
int nc_decode(nc_ctx* ctx, const uint8_t* in, size_t nbytes, int32_t* const* tokens_out,
              int64_t* lens_out);

/* Stream count recorded in a container header (HOST bytes), or NC_ECORRUPT. */
int nc_container_streams(const uint8_t* in, size_t nbytes, int* n_streams);

const char* nc_status_str(int status);
/* Message of the last failing call on ctx (never NULL). */
const char* nc_last_error(const nc_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Building blocks, exposed for parity tests and for callers that drive the
 * coder themselves.
 * ------------------------------------------------------------------------- */

/* CDF quantisation (Sec. 3.3) of n rows of V binary32 probabilities:
 * c_i = max(floor, floor(p_i * (T - V*floor))) with the product taken
 * exactly, the residual T - sum c added to the first maximum of p, then the
 * exclusive prefix sum, cdf[0] = 0, cdf[V] = T.  p DEVICE float[n * V],
 * cdf DEVICE uint32[n * (V + 1)], stream a cudaStream_t or NULL (legacy
 * default stream).  Returns NC_ENUMERIC when a row holds a non-finite or
 * negative value, a value >= 2, or the residual would leave the argmax count
 * below the floor (that row's cdf is then unspecified); NC_EINVAL for bad
 * sizes.  Synchronises the stream. */
int nc_probs_to_cdf(const float* p, int n, int V, int log2_total, uint32_t floor,
                    uint32_t* cdf, void* stream);

/* nc_probs_to_cdf for callers that cannot let a library allocate device
 * memory: for example a process whose allocator already holds all free HBM,
 * a latency-critical loop where a cudaMalloc / cudaFree would synchronise
 * the device, or code sharing a GPU with a framework that owns every
 * allocation.  The paper has no counterpart; it is an interface addition.
 * Same arguments, results and errors as nc_probs_to_cdf, but it calls no
 * cudaMalloc, cudaFree or other allocating routine: the per-row status words
 * live in a fixed device array of NC_NOALLOC_MAX_ROWS int32 that the library
 * image carries, so every GPU that loads the library holds those 16 KB until
 * the process exits.
 *  - n > NC_NOALLOC_MAX_ROWS returns NC_EINVAL (split the rows over calls).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it; make that first call before any
 *    stream capture.  The first call after a reset of the device's context
 *    (cudaDeviceReset) looks it up again.
 *  - Every call, on any stream, shares the one array; each call clears the
 *    words it uses.  Calls whose GPU work overlaps (another host thread, or
 *    another stream) race on it: serialise them.
 *  - Synchronises `stream`. */
#define NC_NOALLOC_MAX_ROWS 4096
int nc_probs_to_cdf_noalloc(const float* p, int n, int V, int log2_total, uint32_t floor,
                            uint32_t* cdf, void* stream);

/* Elementwise exact product floor, c[i] = max(floor, floor(p[i] * K)), for
 * binary32 p[i] in [0, 2) and 0 < K < 2^24 (the quantiser's inner step,
 * Sec. 3.3).  p DEVICE float[n], c DEVICE uint32[n]; entries outside [0, 2)
 * give 0xFFFFFFFF.  Asynchronous on `stream`. */
int nc_floor_counts(const float* p, int64_t n, uint32_t K, uint32_t floor, uint32_t* c,
                    void* stream);

/* One model step like nc_step_cdf that also returns the intermediate
 * distributions of every stream (DEVICE float[n * V] each, any may be NULL):
 * z the logits (Eq. lm), p_tilde the biased LLM distribution (Sec. 3.6),
 * p_ng the N-gram distribution (Sec. 3.4), p the mixed binary32 probabilities
 * handed to the quantiser; cdf_out as in nc_step_cdf. */
int nc_step_probe(nc_ctx* ctx, int n, const int32_t* stream_ids, float* z, float* p_tilde,
                  float* p_ng, float* p, uint32_t* cdf_out);

/* Copy a stream's adaptive state to HOST buffers (any may be NULL): bias
 * float[V] (Sec. 3.6), mixer log-weights float[2] (Sec. 3.5), tokens coded. */
int nc_stream_state(nc_ctx* ctx, int32_t stream_id, float* bias, float* mix_logw,
                    int64_t* n_coded);

/* Tensor-core GEMM (tcgen05, the projections of the batched path):
 * Y[n][m] = sum_k W[m][k] X[n][k] with FP32 accumulation.
 *   W DEVICE [M][K], X DEVICE [N][K]: BF16 (fp8 = 0) or FP8 E4M3 (fp8 = 1),
 *     row-major, 16-byte aligned, K * element size a multiple of 16.
 *   w_scale DEVICE float[M], x_scale DEVICE float[N] (FP8 only): the product
 *     is scaled by w_scale[m] * x_scale[n].
 *   bn: batch tile, 32 | 64 | 128 | 256 (results do not depend on it).
 *   Y DEVICE float[N][M].  Synchronises `stream`.
 * Errors: NC_EINVAL, NC_ENOMEM, NC_ECUDA, NC_ETIMEOUT (a bounded pipeline
 * wait gave up). */
int nc_gemm_tc(const void* W, const void* X, const float* w_scale, const float* x_scale, int fp8, int M,
               int N, int K, int bn, float* Y, void* stream);

/* Diagnostic of the failure path of the device waits: one bounded wait, at
 * most `polls` polls of an mbarrier that nothing arrives on, through the same
 * wait routine and status word as the tensor-core pipelines (the projections'
 * GEMM and the attention).  The wait gives up, and the call reports it as a
 * stalled pipeline is reported: NC_ETIMEOUT, the context poisoned (every
 * later call but nc_ctx_destroy / nc_last_error returns NC_ESTATE).  No GPU
 * fault is involved and the device stays usable; a new context works.
 * The paper has no counterpart.  Errors: NC_EINVAL, NC_ESTATE, NC_ECUDA. */
int nc_selftest_wait(nc_ctx* ctx, uint32_t polls);

/* Diagnostic of the latency floor of the decode step's chain of dependent
 * kernels: a captured CUDA graph of n_links empty kernels of blocks x
 * threads, each launched with programmatic dependent launch and waiting for
 * its predecessor as the step's kernels do, replayed 3 times untimed and
 * `reps` times between CUDA events on device `device`.  *us_per_link (HOST)
 * receives the device time per link in microseconds.  No device memory is
 * allocated.  The paper has no counterpart.
 * Errors: NC_EINVAL (n_links outside 1..4096, blocks outside 1..65535,
 * threads not a multiple of 32 in 32..1024, reps < 1, NULL output), NC_ECUDA. */
int nc_launch_chain_floor(int device, int n_links, int blocks, int threads, int reps, float* us_per_link);

/* 32-bit arithmetic coder (Sec. 3.8) on the host, for callers that produce
 * their own CDFs.  Encode n intervals [lo[i], hi[i]) of a total 2^log2_total
 * (HOST uint32 arrays) into out (HOST, capacity *inout_nbytes; size and the
 * exact bit count returned).  Errors: NC_EINVAL (empty or out-of-range
 * interval, buffer too small: *inout_nbytes then holds the size needed). */
int nc_ac_encode(const uint32_t* lo, const uint32_t* hi, int64_t n, int log2_total,
                 uint8_t* out, size_t* inout_nbytes, uint64_t* nbits);

/* Decode n symbols with one CDF per symbol: cdfs HOST uint32[n * (V + 1)],
 * bits HOST (nbits valid bits, zeros read past the end), symbols HOST int32[n].
 * Errors: NC_EINVAL, NC_ECORRUPT (a CDF that is not a valid CDF). */
int nc_ac_decode(const uint8_t* bits, uint64_t nbits, const uint32_t* cdfs, int V, int64_t n,
                 int log2_total, int32_t* symbols);

/* rANS coder (the ANS coder of Sec. 6) on the host, for callers that produce
 * their own CDFs.  State x in [2^31, 2^63): a symbol [lo, hi) of a total
 * M = 2^log2_total (1..31), f = hi - lo, encodes as
 * x -> floor(x / f) M + (x mod f) + lo after moving the low 32 bits of x out
 * while x >= 2^(63 - log2_total) f, and decodes as x -> f floor(x / M) +
 * (x mod M) - lo, refilling 32 bits while x < 2^31.  The encoder takes the
 * symbols in reverse from x = 2^31 and writes the final state (8 bytes, little-
 * endian) and then the moved-out words (4 bytes each) in the order the decoder
 * reads them.
 * nc_ans_encode: n intervals (HOST uint32 lo, hi) into out (HOST, capacity
 *   *inout_nbytes; the size returned; out == NULL queries it).
 *   Errors: NC_EINVAL (empty or out-of-range interval, buffer too small).
 * nc_ans_decode: n symbols, one CDF per symbol (HOST uint32[n * (V + 1)]),
 *   into symbols HOST int32[n].  Errors: NC_EINVAL, NC_ECORRUPT (a CDF that is
 *   not a valid CDF, a length that is not 8 + 4 k bytes, or a final state
 *   other than 2^31 with every word read). */
int nc_ans_encode(const uint32_t* lo, const uint32_t* hi, int64_t n, int log2_total, uint8_t* out,
                  size_t* inout_nbytes);
int nc_ans_decode(const uint8_t* data, size_t nbytes, const uint32_t* cdfs, int V, int64_t n, int log2_total,
                  int32_t* symbols);

/* File-level chunking (Sec. 3.11) on token ids, for coding one file as up to
 * n_chunks independent streams of one container (nc_encode): cut k of
 * n_chunks - 1 falls just after the first line-ending token at or after
 * position ceil(k n / n_chunks) - 1; cuts without a line end after them, at
 * or before the previous cut, or at n are dropped.
 *   tokens HOST int32[n] in [0, V); is_boundary HOST uint8[V], non-zero for
 *   an id that ends a line (the tokenizer's knowledge, the caller's);
 *   cuts HOST int64[n_chunks + 1] receives 0 = c_0 < ... < c_m = n, and
 *   *n_chunks_out = m (0 for n = 0): chunk j is tokens[c_j, c_{j+1}).
 * Errors: NC_EINVAL (NULL pointers, n_chunks < 1, an id out of range). */
int nc_split_chunks(const int32_t* tokens, int64_t n, const uint8_t* is_boundary, int V, int n_chunks,
                    int64_t* cuts, int* n_chunks_out);

/* NC06 hybrid binary format (Sec. 3.10): the runs of text (kind 0) and
 * binary (kind 1) bytes of an arbitrary byte string, alternating.  Bytes are
 * text-like when printable ASCII (32..126), tab, LF or CR; text runs shorter
 * than 64 bytes become binary; binary gaps of at most 8 bytes between two
 * text runs become text; binary runs shorter than 64 bytes next to a text
 * run become text (the four rules in the order listed; adjacent runs of one
 * kind merge after each).  Text runs are coded as the streams of one
 * NC05 container, binary runs concatenated into one blob.
 *   data HOST uint8[n]; kinds HOST uint8[cap], lens HOST int64[cap] receive
 *   the runs in order, *n_runs their count.  cap = 0 queries the count only.
 * Errors: NC_EINVAL (NULL pointers, n < 0, cap below the count). */
int nc_hybrid_segments(const uint8_t* data, int64_t n, uint8_t* kinds, int64_t* lens, int64_t cap,
                       int64_t* n_runs);

/* Assemble an NC06 container into HOST out (size query when out is NULL,
 * as nc_encode): "NC06", version 1, a flags byte and the temperature
 * (binary16), the run count (u32), per run its kind (u8) and length (u32),
 * the binary blob's method (u8: 0 raw, 1 gzip, 2 LZMA; the caller
 * compresses) and stored length (u32), the stored blob, then `text`, the
 * NC05 container of the text runs' streams (nc_encode), empty when there is
 * no text run.  The flags byte and temperature are that container's (a
 * decoder replays them); without text runs, 0 and 1.0.  Little-endian.
 * Errors: NC_EINVAL (NULL pointers, a kind other than 0 / 1, a length
 * outside [1, 2^32), a method other than 0..2, a blob of 2^32 bytes or more,
 * a non-empty text that is not an NC05 container, out too small:
 * *inout_nbytes then holds the size needed). */
int nc_hybrid_pack(const uint8_t* kinds, const int64_t* lens, int64_t n_runs, int method, const uint8_t* stored,
                   size_t n_stored, const uint8_t* text, size_t n_text, uint8_t* out, size_t* inout_nbytes);

/* Read an NC06 container (HOST buf[n]): the runs as nc_hybrid_segments
 * gives them (cap = 0: count only), the blob's method, the stored blob at
 * buf[*stored_off .. + *stored_len), the text runs' NC05 container from
 * buf[*text_off] to the end.  Errors: NC_ECORRUPT (not an NC06 version 1
 * container, a bad run or method, a truncated section), NC_EINVAL (NULL
 * pointers, cap below the count). */
int nc_hybrid_parse(const uint8_t* buf, size_t n, uint8_t* kinds, int64_t* lens, int64_t cap, int64_t* n_runs,
                    int* method, size_t* stored_off, size_t* stored_len, size_t* text_off);

/* Mixed-distribution NLL L = -log(w0 p_tilde(t*) + w1 p_ng(t*)), w = softmax(theta),
 * p_tilde = softmax(z / tau + b), for n rows (the differentiable update rule).
 *   z, b, p_ng DEVICE float[n * V]; theta DEVICE float[n * 2]; target DEVICE int32[n];
 *   warm DEVICE int32[n] (non-zero: p = p_tilde, the warm-up case);
 *   loss DEVICE float[n].  Asynchronous on `stream`. */
int nc_mix_nll_fwd(const float* z, const float* b, const float* p_ng, const float* theta,
                   const int32_t* target, const int32_t* warm, int n, int V, float tau,
                   float* loss, void* stream);

/* Gradient of nc_mix_nll_fwd's loss scaled by gout (DEVICE float[n], NULL = 1):
 * db DEVICE float[n * V] = gout * rho * (p_tilde - e_t*), rho = w0 p_tilde(t*)/p_mix(t*)
 * (1 in warm-up); dtheta DEVICE float[n * 2] = gout * (w - w * p_j(t*)/p_mix(t*))
 * (0 in warm-up).  Deterministic (no atomics).  Asynchronous on `stream`. */
int nc_mix_nll_bwd(const float* z, const float* b, const float* p_ng, const float* theta,
                   const int32_t* target, const int32_t* warm, const float* gout, int n, int V,
                   float tau, float* db, float* dtheta, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NC24_H */
