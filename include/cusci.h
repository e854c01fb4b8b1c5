/*
 * cusci.h -- C ABI of libcusci: coupled-configuration generation with
 * Slater-Condon matrix elements, |H_ij| screening, in-batch de-duplication and
 * the variational energy with its adjoint, for selected configuration
 * interaction driven by neural-network quantum states (NNQS-SCI, Stage 1 and
 * Stage 3 of the paper's pipeline, Sec. 3; kernels of Sec. 4.1-4.2).
 *
 * Data model (Sec. 2.1; the paper fixes no spin-orbital order, this library
 * takes the interleaved one):
 *   - norb spatial orbitals, M = 2*norb spin orbitals, spin orbital
 *     s = 2*p + sigma with sigma = 0 for alpha, 1 for beta.
 *   - A determinant is W = ceil(M/64) little-endian uint64 words; spin orbital
 *     s is bit (s & 63) of word (s >> 6).  W is 1 or 2 (norb <= 64).
 *   - Arrays of determinants are row-major [n][W].  "Sorted" means ascending as
 *     W-word unsigned integers, word W-1 most significant.
 *   - Integrals are real: h1[p*norb+q] symmetric, h2 in chemists' notation,
 *     h2[((p*norb+q)*norb+r)*norb+s] = (pq|rs) with the 8-fold symmetry.
 *   - H = Ecore + sum h_pq a+_{p s} a_{q s}
 *           + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s};
 *     a_s and a+_s carry the phase (-1)^(occupied spin orbitals below s).
 *
 * Coupled set C_i of a source determinant (Sec. 2.1: every j with H_ij != 0,
 * reached by moving one or two electrons, j = i included), in canonical order:
 * the diagonal first (always kept); then singles i->a with occupied i
 * ascending and same-spin virtual a ascending; then doubles with occupied pairs
 * i<j lexicographic and (a,b) lexicographic (a<b when i and j share a spin, a of
 * i's spin and b of j's spin otherwise).  Off-diagonal entries are kept iff
 * |H_ij| > eps (the screening test of Algorithm 1; eps < 0 keeps all).
 * Matrix elements are FP64 and bit-identical to the Slater-Condon closed forms
 * summed in the order: diagonal (Ecore + sum_i h_ii) + sum_{i<j}[(ii|jj) -
 * same-spin (ij|ji)]; single h_ai then, for k in O ascending (k != i), +(ai|kk)
 * and, for k of a's spin, -(ak|ki); double (ai|bj) - (aj|bi) for a same-spin
 * pair, (ai|bj) otherwise.
 *
 * Conventions of every call:
 *   - The caller owns every buffer it passes (device pointers are prefixed d_,
 *     host pointers h_); the library owns only cusci_system objects and what
 *     they hold.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated.
 *   - Nothing aborts or traps.  Every call returns a status; the message of the
 *     last failure on the calling thread is cusci_last_error().
 *   - A cusci_system may be used from several streams only if the calls are
 *     ordered between them by the caller (its screening-mask cache is shared).
 *   - Requires a GPU of compute capability 10.3 (the library is built for
 *     sm_103a only).
 */
#ifndef CUSCI_H
#define CUSCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CUSCI_OK = 0,
    CUSCI_ERR_INVALID = 1,     /* bad argument or precondition violated          */
    CUSCI_ERR_OOM = 2,         /* device / host allocation or workspace too small */
    CUSCI_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
    CUSCI_ERR_OVERFLOW = 4,    /* output capacity / offsets inconsistent          */
    CUSCI_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up              */
    CUSCI_ERR_UNSUPPORTED = 6  /* size outside what this build handles            */
} cusci_status;

typedef struct cusci_system cusci_system; /* opaque, library-owned */

/* Message of the last failing call on this thread ("" if none). */
const char *cusci_last_error(void);
/* Library version string. */
const char *cusci_version(void);
/* Number of kernels the library has launched in this process so far (host-side
 * count of successful launches, all devices and streams). */
uint64_t cusci_kernel_launches(void);
/* Per-kernel timing of the sample-sort de-duplication (diagnostics; the
 * regular-sampling partition of Sec. 4.1.1).  cusci_set_kernel_timing(1)
 * resets the record and makes every later cusci_dedup call on that path (up to
 * 64 calls, on the current device) record a CUDA event on its own stream
 * before its first kernel and after each of its phases; 0 stops recording.
 * cusci_dedup_phase_ms waits for the recorded events and writes, for phase
 * i < min(max, number of phases), the summed milliseconds of all recorded
 * calls to h_ms[i] (host array); *h_calls (nullable) receives the number of
 * calls summed.  Returns the number of phases written.  Phase names come from
 * cusci_dedup_phase_name(i) (static strings; NULL out of range).  Timing adds
 * no synchronisation to the calls themselves. */
cusci_status cusci_set_kernel_timing(int on);
int cusci_dedup_phase_ms(double *h_ms, int max, int *h_calls);
const char *cusci_dedup_phase_name(int i);

/* ------------------------------------------------------------------ system
 * Builds the device-side integral tables of one molecular system (the
 * excitation tables T_single / T_double of Sec. 4.2.1, held here as permuted
 * FP64 slabs plus per-eps screening bitmasks).  h1: host, norb*norb doubles.
 * h2: host, norb^4 doubles.  Both are copied; the caller may free them on
 * return.  1 <= norb <= 64, 0 <= n_alpha, n_beta <= norb.  Synchronous.
 * The system caches the screening masks of the four most recently used eps
 * values; a call at a fifth eps rebuilds the least recently used set in place
 * after waiting for all earlier work on the device (calls on other streams may
 * still read it), and fails with CUSCI_ERR_INVALID if its stream is being
 * captured into a CUDA graph (run each eps once before capturing).
 * Errors: CUSCI_ERR_INVALID (sizes), CUSCI_ERR_OOM, CUSCI_ERR_CUDA. */
cusci_status cusci_system_create(int norb, int n_alpha, int n_beta, const double *h1,
                                 const double *h2, double ecore, cusci_system **out);
void cusci_system_destroy(cusci_system *sys);
/* W of the system's determinants (1 or 2); 0 for NULL. */
int cusci_system_words(const cusci_system *sys);

/* ------------------------------------------------------------------ generation
 * Count pass (the "count" half of count-then-fill, Sec. 4.2.2; it replaces the
 * g_counter slab reservation of Algorithm 1).
 * d_dets: device [n][W] sources.  Bits at or above M are ignored; the coupled
 * set is that of the occupation the bits describe (use cusci_check_dets to
 * enforce the system's electron counts).  d_counts: device int64[n], receives
 * |C_i| after screening, diagonal included.  n == 0 is a no-op. */
cusci_status cusci_count_coupled(const cusci_system *sys, const uint64_t *d_dets, int64_t n,
                                 double eps, int64_t *d_counts, void *stream);

/* Exclusive prefix sum: d_offsets[0] = 0, d_offsets[k+1] = d_offsets[k] +
 * d_counts[k] (device int64, n+1 entries, so d_offsets[n] is the total).
 * Workspace: cusci_scan_workspace bytes of device memory, 8-byte aligned. */
cusci_status cusci_scan_workspace(int64_t n, size_t *bytes);
cusci_status cusci_exclusive_scan(const int64_t *d_counts, int64_t n, int64_t *d_offsets,
                                  void *d_ws, size_t ws_bytes, void *stream);

/* Exclusive prefix sum that allocates nothing.  The paper has no counterpart;
 * it exists for callers that cannot allocate device memory or pass a
 * workspace: code inside a framework that has reserved the device's memory for
 * its own pool, latency-critical loops where cudaMalloc's implicit device
 * synchronisation would stall other streams, and bindings that can only pass
 * pointers to existing buffers.  Same result as cusci_exclusive_scan.
 * Scratch: a fixed array inside the library (512 KiB per device, held by every
 * device that loads the library until the process exits); n is limited to
 * cusci_scan_static_max() counts (134,217,728), larger n returns
 * CUSCI_ERR_UNSUPPORTED.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress, with the device current), so make that
 * first call before any stream capture.  All calls share the one array: calls
 * that overlap on the GPU (other streams, other threads) race and must be
 * ordered by the caller.  Calls no cudaMalloc, cudaFree or allocating routine. */
int64_t cusci_scan_static_max(void);
cusci_status cusci_exclusive_scan_static(const int64_t *d_counts, int64_t n, int64_t *d_offsets,
                                         void *stream);

/* Fill pass (Algorithm 1 and Sec. 4.2.2): writes C_i to rows
 * [d_offsets[i], d_offsets[i+1]) of d_out_dets (device [total][W]) and d_out_h
 * (device double[total]) in canonical order.  d_offsets must be the exclusive
 * scan of the counts of the same sources at the same eps; a row range that
 * does not match the regenerated count is reported through d_status.
 * d_status: device int32 (nullable); set to CUSCI_ERR_OVERFLOW if any source's
 * range disagrees (the rows of such a source are then left partly unwritten),
 * untouched otherwise. */
cusci_status cusci_gen_coupled(const cusci_system *sys, const uint64_t *d_dets, int64_t n,
                               double eps, const int64_t *d_offsets, uint64_t *d_out_dets,
                               double *d_out_h, int32_t *d_status, void *stream);

/* Validates sources: d_status (device int32) is set to CUSCI_ERR_INVALID if any
 * row has the wrong alpha/beta electron counts or a bit at or above M,
 * untouched otherwise. */
cusci_status cusci_check_dets(const cusci_system *sys, const uint64_t *d_dets, int64_t n,
                              int32_t *d_status, void *stream);

/* ------------------------------------------------------------------ de-duplication
 * In-batch de-duplication (Sec. 4.1 local sort + unique; Sec. 3 reverse index):
 * d_unique receives the sorted distinct keys (capacity total*W words),
 * d_inverse[k] the position of key k in d_unique (int32 if index_bytes == 4,
 * int64 if 8; int32 requires total < 2^31).  n_ones >= 0 declares that every
 * key has exactly n_ones set bits among its low n_bits bits, which lets the
 * sort run on the keys' combinatorial rank (fewer radix passes); n_ones < 0
 * sorts the raw low n_bits bits.  1 <= n_bits <= 64*W, W in {1,2}.
 * d_n_unique: device int64 receiving the distinct count.  h_n_unique: host,
 * nullable; if given, the call synchronizes the stream and writes it there.
 * d_status: device int32, nullable: CUSCI_ERR_INVALID if a key breaks the
 * n_ones declaration (outputs then undefined).
 * Workspace: cusci_dedup_workspace bytes of device memory, 256-byte aligned. */
cusci_status cusci_dedup_workspace(int64_t total, int W, int n_bits, int n_ones, size_t *bytes);
cusci_status cusci_dedup(const uint64_t *d_keys, int64_t total, int W, int n_bits, int n_ones,
                         void *d_ws, size_t ws_bytes, uint64_t *d_unique, void *d_inverse,
                         int index_bytes, int64_t *d_n_unique, int64_t *h_n_unique,
                         int32_t *d_status, void *stream);

/* ------------------------------------------------------------------ energy
 * Variational energy over a selected set S (Eq. 1 restricted to S, Sec. 2.1;
 * Stage 3 of Sec. 3): (H psi)_i = sum over j in C_i(eps) with j in S of
 * H_ij psi_j, E = psi.(H psi) / psi.psi.  The coupled lists are regenerated,
 * never stored (the just-in-time reverse index of Sec. 4.3).
 * d_S: device [nS][W], strictly ascending, nS >= 1.  d_psi: device double[nS].
 * d_E, d_norm2: device double[1].  d_Hpsi: device double[nS], nullable (H psi
 * is then kept only in the workspace).  d_status (device int32, nullable): set
 * to CUSCI_ERR_INVALID if S is not strictly ascending (results then undefined).
 * Workspace: cusci_energy_workspace bytes of device memory, 256-byte aligned;
 * it holds a hash table of S and is overwritten by every call.
 * The reductions are deterministic (fixed order, no atomics). */
cusci_status cusci_energy_workspace(const cusci_system *sys, int64_t nS, size_t *bytes);
cusci_status cusci_energy_fwd(const cusci_system *sys, const uint64_t *d_S, int64_t nS,
                              const double *d_psi, double eps, double *d_E, double *d_norm2,
                              double *d_Hpsi, void *d_ws, size_t ws_bytes, int32_t *d_status,
                              void *stream);
/* Adjoint (Sec. 3 Stage 3, backpropagation of the energy):
 * d_grad[i] = g * 2 ((H psi)_i - E psi_i) / norm2, with E and norm2 from the
 * forward call and g = *d_grad_out (device double; NULL means 1).  d_Hpsi may
 * be NULL, in which case H psi is recomputed from the coupled lists. */
cusci_status cusci_energy_bwd(const cusci_system *sys, const uint64_t *d_S, int64_t nS,
                              const double *d_psi, double eps, const double *d_E,
                              const double *d_norm2, const double *d_Hpsi,
                              const double *d_grad_out, double *d_grad, void *d_ws,
                              size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ local energy
 * The SCI energy in the paper's local form (Eq. 5; Stage 3 of Sec. 3): over the
 * coupled lists of the sources (CSR d_offsets[n+1], elements d_h) and the
 * reverse index d_inverse into the distinct coupled set U (both as written by
 * cusci_gen_coupled and cusci_dedup), with amplitudes d_psi_u on U:
 *   y_i = sum_{e in row i} H_e psi_u[inverse[e]],  psi_i = psi_u[inverse[offsets[i]]]
 *   E = sum_i psi_i y_i / sum_i psi_i^2.
 * Every row must start with its diagonal (the source itself) and every inverse
 * value must lie in [0, n_unique).  d_y: device double[n], nullable.  d_E,
 * d_norm2: device double[1].  The forward reduction is deterministic.
 * Workspace: cusci_local_energy_workspace bytes, 256-byte aligned. */
cusci_status cusci_local_energy_workspace(int64_t n, size_t *bytes);
cusci_status cusci_local_energy_fwd(const int64_t *d_offsets, int64_t n, const double *d_h,
                                    const void *d_inverse, int index_bytes,
                                    const double *d_psi_u, double *d_y, double *d_E,
                                    double *d_norm2, void *d_ws, size_t ws_bytes, void *stream);
/* Adjoint: d_grad_u[u] = g ( sum_{e: inverse[e]=u} psi_{i(e)} H_e
 *   + sum_{rows i whose source is u} (y_i - 2 E psi_i) ) / norm2, g = *d_grad_out
 * (NULL: 1).  d_y from the forward call, or NULL to recompute it.  The
 * scatter-add runs in 128-bit fixed point (integer atomics), so the gradient
 * is bit-reproducible run to run and exact up to a 2^-64 truncation per term.
 * Workspace: cusci_local_energy_bwd_workspace(n, n_unique) bytes, 256-byte
 * aligned (16 bytes per distinct configuration plus the rows' scratch). */
cusci_status cusci_local_energy_bwd_workspace(int64_t n, int64_t n_unique, size_t *bytes);
cusci_status cusci_local_energy_bwd(const int64_t *d_offsets, int64_t n, const double *d_h,
                                    const void *d_inverse, int index_bytes,
                                    const double *d_psi_u, int64_t n_unique, const double *d_y,
                                    const double *d_E, const double *d_norm2,
                                    const double *d_grad_out, double *d_grad_u, void *d_ws,
                                    size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ regular-sampling partition
 * Steps 1 and 2 of the paper's distributed de-duplication (Sec. 4.1.1, Fig. 3)
 * for P ranks.  d_keys: device [*][W]; run r (rank r's locally sorted distinct
 * keys) is rows [d_run_offsets[r], d_run_offsets[r+1]) (device int64[P+1]).
 * Each non-empty run contributes S samples at positions floor(k |run| / S),
 * k < S; the samples are sorted and splitter j (j < P-1) is the sample at
 * position ((j+1) * count) / P - 1 (count = number of samples), written to
 * d_splitters (device [P-1][W]).  d_bounds (device int64 [P][P+1]) receives the
 * cuts: rank q's share of run r is rows [bounds[r][q], bounds[r][q+1]), the keys
 * k with splitter[q-1] < k <= splitter[q].  P * S * W must not exceed 16384
 * (next power of two).  Step 3 (exchange and final merge) is
 * cusci_partition_exchange, one cusci_dedup and cusci_partition_split. */
cusci_status cusci_partition_plan(const uint64_t *d_keys, int W, const int64_t *d_run_offsets,
                                  int P, int S, uint64_t *d_splitters, int64_t *d_bounds,
                                  void *stream);
/* Step 1 of the same de-duplication for P ranks on one GPU (Sec. 4.1.1): rank r
 * owns entries [d_entry_offsets[r], d_entry_offsets[r+1]) (device int64[P+1],
 * non-decreasing, [0] = 0, [P] = total) of d_keys (device [total][W], keys
 * below 2^n_bits).  d_joint (device [total][W]) receives every key with its
 * owner rank written into bits [n_bits, n_bits + ceil(log2 P)), so that one
 * cusci_dedup of d_joint (n_bits + ceil(log2 P) bits, n_ones = -1) yields all
 * ranks' locally sorted distinct runs, in rank order.  A key with a bit at or
 * above n_bits sets *d_status (nullable) to CUSCI_ERR_INVALID.  1 <= P <= 1024;
 * CUSCI_ERR_UNSUPPORTED when n_bits + ceil(log2 P) > 64 W.  Asynchronous. */
cusci_status cusci_rank_join(const uint64_t *d_keys, int W, int64_t total,
                             const int64_t *d_entry_offsets, int P, int n_bits,
                             uint64_t *d_joint, int32_t *d_status, void *stream);
/* The runs of Step 1 out of the sorted distinct joined keys: d_runs (device
 * [capacity][W]) receives the first *d_n_unique keys (a device count, e.g.
 * from cusci_dedup) with the rank bits cleared; d_run_offsets (device
 * int64[P+1]) the start of every rank's run ([P] = *d_n_unique).  Same P and
 * n_bits as cusci_rank_join.  Asynchronous. */
cusci_status cusci_rank_runs(const uint64_t *d_joint_unique, int W, const int64_t *d_n_unique,
                             int64_t capacity, int P, int n_bits, uint64_t *d_runs,
                             int64_t *d_run_offsets, void *stream);
/* Step 3's all-to-all on one GPU (Sec. 4.1.1, Fig. 3): rank q receives, in
 * rank order r = 0..P-1, rows [d_bounds[r][q], d_bounds[r][q+1]) of d_runs
 * (the cuts of cusci_partition_plan, device int64 [P][P+1]).  Rank q's rows are
 * written to d_recv (device, rows >= the runs' total) from row
 * d_recv_offsets[q]; d_recv_offsets (device int64[P+1]) is written here,
 * [P] = rows received in all.  One block per (q, r) segment.  Asynchronous. */
cusci_status cusci_partition_exchange(const uint64_t *d_runs, int W, int P,
                                      const int64_t *d_bounds, uint64_t *d_recv,
                                      int64_t *d_recv_offsets, void *stream);
/* Final partitions: the ranks' key ranges are disjoint, so one cusci_dedup of
 * all received rows is every rank's final sort + unique at once; this cuts its
 * output d_unique (device [*][W], *d_n_unique rows) at the P-1 splitters:
 * d_part_offsets (device int64[P+1]) receives for q = 1..P-1 the number of
 * distinct keys <= splitter[q-1], [0] = 0 and [P] = *d_n_unique.
 * Asynchronous. */
cusci_status cusci_partition_split(const uint64_t *d_unique, int W, const int64_t *d_n_unique,
                                   const uint64_t *d_splitters, int P, int64_t *d_part_offsets,
                                   void *stream);

/* ------------------------------------------------------------------ reverse index
 * Just-in-time reverse index (Stage 3 of Sec. 3, Sec. 4.3.4): d_inverse[k] =
 * position of key k (device [n][W]) in the sorted distinct set d_unique
 * (device [n_unique][W], as written by cusci_dedup or cusci_stream_gen_dedup),
 * or -1 with d_status (device int32, nullable) set to CUSCI_ERR_INVALID if the
 * key is absent.  index_bytes 4 or 8.  n_unique <= 2^29 (W = 1) or 2^28
 * (W = 2).  Meant for batches of a host-resident coupled set streamed in. */
cusci_status cusci_reverse_index(const uint64_t *d_unique, int64_t n_unique, int W,
                                 const uint64_t *d_keys, int64_t n, void *d_inverse,
                                 int index_bytes, int32_t *d_status, void *stream);
/* The same reverse index through a hash table of the distinct set, built once
 * and then probed by every batch (about one random access per key instead of
 * a search).  cusci_reverse_table_bytes: bytes of the table for n_unique keys
 * of W words (a power of two of at least 1.5 n_unique slots; key words, then
 * an int64 position per slot).  cusci_reverse_table_build fills the caller's
 * d_table (device, 16-byte aligned, >= that many bytes) from d_unique (device
 * [n_unique][W], distinct keys; asynchronous; d_status set to
 * CUSCI_ERR_OVERFLOW if a key found no slot, which the sizing rules out).
 * cusci_reverse_index_table: d_inverse[k] = position of key k in d_unique,
 * or -1 with d_status (nullable) set to CUSCI_ERR_INVALID when absent; same
 * n_unique and W as the build; index_bytes 4 or 8.  Asynchronous. */
cusci_status cusci_reverse_table_bytes(int64_t n_unique, int W, size_t *bytes);
cusci_status cusci_reverse_table_build(const uint64_t *d_unique, int64_t n_unique, int W,
                                       void *d_table, size_t table_bytes, int32_t *d_status,
                                       void *stream);
cusci_status cusci_reverse_index_table(const void *d_table, int64_t n_unique, int W,
                                       const uint64_t *d_keys, int64_t n, void *d_inverse,
                                       int index_bytes, int32_t *d_status, void *stream);

/* ------------------------------------------------------------------ top-K selection
 * Streaming two-level top-K (Stage 2 of Sec. 3, the running best set of
 * Sec. 4.3.4): merges one batch (d_scores / d_ids, device, n items; scores
 * non-negative FP64, ids distinct) into the running best set d_best_scores /
 * d_best_ids (device, capacity K, count in device int64 *d_best_count; start
 * it at 0).  The batch's own K best are selected first, then merged with the
 * running set.  Best = larger score, equal scores by smaller id (exact and
 * deterministic); the running set is kept unordered; -0.0 counts as 0.
 * d_status (device int32, nullable): set to CUSCI_ERR_INVALID if a score of the
 * batch is negative or NaN (the selection is then not meaningful).
 * Workspace: cusci_topk_workspace(n, K) bytes, 256-byte aligned.  No host
 * synchronisation. */
cusci_status cusci_topk_workspace(int64_t batch, int64_t K, size_t *bytes);
cusci_status cusci_topk_update(const double *d_scores, const int64_t *d_ids, int64_t n, int64_t K,
                               double *d_best_scores, int64_t *d_best_ids,
                               int64_t *d_best_count, void *d_ws, size_t ws_bytes,
                               int32_t *d_status, void *stream);

/* ------------------------------------------------------------------ streaming
 * Generation + de-duplication in mini-batches out of a caller-owned device
 * pool (Sec. 4.3: mini-batch execution, compute/transfer overlap, Stage 1
 * offload of the original coupled set to host memory).
 * h_dets: host [n][W] sources.  d_pool: device memory of pool_bytes, 256-byte
 * aligned, at least cusci_stream_pool_bytes(); the library uses nothing else
 * on the device.  The pool holds the per-source arrays, a hash set of the
 * distinct keys (at most 3/4 full at unique_capacity) and the two batch
 * buffers; the final sort of the distinct keys then reuses the hash set's
 * memory.  batch_entries: capacity of one mini-batch (two are in flight:
 * one filled while the other is copied out); every single source's list must
 * fit one batch.  h_offsets: host int64[n+1], receives the CSR offsets of the
 * whole coupled set.  h_out_dets / h_out_h: host sinks (pinned for overlap)
 * of host_capacity entries receiving the coupled lists in canonical order, or
 * both NULL to skip the offload.  d_unique: device [unique_capacity][W],
 * receives the sorted distinct targets of all batches; *h_n_unique their
 * number.  h_stats (nullable, host int64[6]): total entries, batches, peak pool
 * bytes used, bytes offloaded, microseconds spent up to the last batch's
 * offload (counts, batches, hash inserts, copies) and in the final sort of the
 * distinct keys.  Synchronous (returns when everything landed).
 * Errors: CUSCI_ERR_OOM (pool or sinks too small, or a source longer than a
 * batch), CUSCI_ERR_OVERFLOW (more distinct keys than unique_capacity),
 * CUSCI_ERR_TIMEOUT (a bounded wait in the hash set gave up),
 * CUSCI_ERR_UNSUPPORTED (64 or more electrons). */
/* The streaming path's device hash set, exposed so that its bounded wait can
 * be exercised (the failure tier of the tests; no counterpart in the paper).
 * Inserts the n keys d_keys (device [n][W]) into d_table (device [slots][W],
 * slots a power of two, empty slots all ones) by open addressing; *d_n_new
 * (device, accumulated) counts keys not present before.  A two-word insert
 * that finds its first word already claimed polls the slot's second word at
 * most spin_limit times (the streaming path uses 2^20); if it is still empty
 * then, d_status (device int32, nullable) receives CUSCI_ERR_TIMEOUT and the
 * key is dropped -- no wait is unbounded.  A full table gives
 * CUSCI_ERR_OVERFLOW.  Asynchronous on the stream. */
cusci_status cusci_hash_insert_probe(const uint64_t *d_keys, int64_t n, int W, uint64_t *d_table,
                                     int64_t slots, int spin_limit, unsigned long long *d_n_new,
                                     int32_t *d_status, void *stream);
cusci_status cusci_stream_pool_bytes(const cusci_system *sys, int64_t n_sources,
                                     int64_t batch_entries, int64_t unique_capacity,
                                     size_t *bytes);
cusci_status cusci_stream_gen_dedup(const cusci_system *sys, const uint64_t *h_dets, int64_t n,
                                    double eps, void *d_pool, size_t pool_bytes,
                                    int64_t batch_entries, int64_t *h_offsets,
                                    uint64_t *h_out_dets, double *h_out_h,
                                    int64_t host_capacity, uint64_t *d_unique,
                                    int64_t unique_capacity, int64_t *h_n_unique,
                                    int64_t *h_stats, void *stream);

/* ------------------------------------------------------------------ batched systems
 * Many independent systems in one persistent launch (the persistent
 * grid-stride kernel of Algorithm 1, extended over systems): warps pull
 * (system, source chunk) work items, largest estimated cost first, from an
 * atomic counter.  Sources of every system are stored as two words per
 * determinant, systems back to back in the order given (one-word systems carry
 * a zero high word); targets are written the same way into one CSR over all
 * sources.  cusci_batch_create: systems stay owned by the caller and must
 * outlive the batch; h_sources[k] = number of sources of system k; chunk =
 * sources per work item (cusci_batch_set_chunk changes it).  The batch owns
 * its own screening masks, one set per system, so calls on the systems
 * themselves never change what a batch launch (or a graph replay of one)
 * reads.  The first count or gen call at a new eps synchronizes the stream and
 * rebuilds those masks; later calls at the same eps are plain asynchronous
 * launches (capturable in a CUDA graph).  Per-system de-duplication is
 * cusci_dedup on each system's slice of the targets. */
typedef struct cusci_batch cusci_batch;
cusci_status cusci_batch_create(const cusci_system *const *systems, int n_systems,
                                const int64_t *h_sources, int chunk, cusci_batch **out);
void cusci_batch_destroy(cusci_batch *batch);
cusci_status cusci_batch_set_chunk(cusci_batch *batch, int chunk);
int64_t cusci_batch_sources(const cusci_batch *batch);
/* d_dets: device [total sources][2]; d_counts: device int64[total sources]. */
cusci_status cusci_batch_count(cusci_batch *batch, const uint64_t *d_dets, double eps,
                               int64_t *d_counts, void *stream);
/* d_offsets: exclusive scan of the counts (total sources + 1); d_out_dets:
 * device [total][2], 16-byte aligned; d_out_h: device double[total];
 * d_status (nullable): CUSCI_ERR_OVERFLOW if offsets and regenerated counts
 * disagree. */
cusci_status cusci_batch_gen(cusci_batch *batch, const uint64_t *d_dets, double eps,
                             const int64_t *d_offsets, uint64_t *d_out_dets, double *d_out_h,
                             int32_t *d_status, void *stream);
/* Blocks per SM of the persistent count / fill grid (1..32; default 8), the
 * second knob of the batch's autotuner beside the work-item size. */
cusci_status cusci_batch_set_grid(cusci_batch *batch, int blocks_per_sm);
/* De-duplication of every system's targets in one pass (the in-batch
 * de-duplication of Sec. 4.1, per system, over the whole batch): target e of
 * system k becomes base_k + its combinatorial rank among the C(M_k, n_k)
 * determinants of system k -- an order-preserving 64-bit key whose ranges are
 * disjoint and in system order -- so one sort yields all systems' sorted
 * distinct sets.  d_offsets / d_targets as written by cusci_batch_gen (total
 * entries).  Outputs per system k, whose entries are
 * [d_offsets[first source of k], d_offsets[first source of k+1]): its sorted
 * distinct targets at the same positions of d_unique (device [total][2]), the
 * id of every entry's target within them in d_inverse (device int32[total]),
 * their number in d_n_unique[k] (device int64[n_systems]).  d_status (device
 * int32, nullable): CUSCI_ERR_INVALID if a target has the wrong electron count
 * or bits above M.  Asynchronous; the number of launches does not depend on
 * the number of systems.  Errors: CUSCI_ERR_UNSUPPORTED if the systems' rank
 * spaces sum to 2^64 or more, or total >= 2^31; CUSCI_ERR_OOM (workspace).
 * Workspace: cusci_batch_dedup_workspace(batch, total) bytes, 256-byte aligned. */
cusci_status cusci_batch_dedup_workspace(const cusci_batch *batch, int64_t total, size_t *bytes);
cusci_status cusci_batch_dedup(cusci_batch *batch, const int64_t *d_offsets,
                               const uint64_t *d_targets, int64_t total, void *d_ws,
                               size_t ws_bytes, uint64_t *d_unique, int32_t *d_inverse,
                               int64_t *d_n_unique, int32_t *d_status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CUSCI_H */
