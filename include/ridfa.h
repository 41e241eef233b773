/*
 * ridfa.h -- C ABI of the GB300 RID recognizer (reduced-interface DFA, speculative
 * data-parallel recognition of regular texts).
 *
 * Method: A. Borsotti, L. Breveglieri, S. Crespi Reghizzi, A. Morzenti, "Minimizing
 * speculation overhead in a parallel recognizer for regular texts" (arXiv 2412.14975).
 *   - chunk automaton B (RI-DFA) built from the position NFA of the RE ............ Sec. 3.1
 *   - chunking x = y_1 ... y_c, y_i non-empty ...................................... Sec. 2
 *   - reach phase: lambda_i(a) = delta^B(a, y_i) for every interface state a ......... Sec. 3.2
 *   - interface function if / if_min, join, acceptance PLAS_c n F^RID != {} ....... Sec. 3.2, 3.4
 *   - all-states DFA comparator (the DFA variant of the classic algorithm) ........ Sec. 2, Fig. 2
 *
 * Conventions shared by every entry point:
 *   - All functions return an int status: RIDFA_OK (0) or a negative RIDFA_E_* code.  No C++
 *     exception crosses this boundary.  ridfa_strerror() names a code.
 *   - Text and chunk-map buffers passed as d_* are DEVICE pointers owned by the caller (e.g. the
 *     data_ptr() of a CUDA tensor); h_* are host pointers owned by the caller.  The library owns
 *     a ridfa_program (host tables, device tables and device scratch) until ridfa_free().
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Device work
 *     is enqueued on it; the *_async calls do not synchronise, the others do.
 *   - Calls that use the same program must not run concurrently on different streams: the
 *     program's device scratch is shared by its calls.
 *   - Chunk boundaries are b_i = floor(i * len / n_chunks), chunk i = text[b_i, b_{i+1}), so
 *     1 <= n_chunks <= len is required (every chunk non-empty, Sec. 2).
 *   - Chunk maps are uint16 [n_chunks][k] (row-major); entry [i][a] is the state reached from
 *     interface slot a over chunk i, or RIDFA_UNDEF (0xFFFF) when the run dies (the undefined
 *     transition).  Row 0 is computed for every slot too, although the join uses only the slot
 *     of {q0} there.
 *
 * RE dialect (bytes, full-text match): literal bytes; '.' any byte; [..] and [^..] with ranges;
 * escapes \n \t \r \xHH and \c for any other c; ( ) grouping, () the empty word; postfix
 * * + ? {m} {m,} {m,n}; concatenation; | (an empty alternative is the empty word).  Bounded
 * repeats expand as r{m,n} = r^m (r(r(...r)?)?)? (n-m nested optional copies).
 */
#ifndef RIDFA_H
#define RIDFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RIDFA_OK 0
#define RIDFA_E_ARG (-1)             /* bad argument (NULL pointer, zero length where not allowed) */
#define RIDFA_E_SYNTAX (-2)          /* the RE does not parse */
#define RIDFA_E_TOO_MANY_STATES (-3) /* RI-DFA (or minimal DFA) exceeds max_states (<= 65534) */
#define RIDFA_E_CHUNKS (-4)          /* n_chunks == 0 or n_chunks > len */
#define RIDFA_E_NOMEM (-5)           /* host or device allocation failed */
#define RIDFA_E_CUDA (-6)            /* a CUDA runtime call failed (no device, launch error, ...) */
#define RIDFA_E_TIMEOUT (-7)         /* a bounded device wait gave up */
#define RIDFA_E_BUSY (-8)            /* admission refused (device-memory budget) */
#define RIDFA_E_UNSUPPORTED (-9)     /* e.g. more interface slots than the kernels support */
#define RIDFA_E_NO_DFA (-10)         /* the program was compiled without the DFA comparator */
#define RIDFA_E_STATE (-11)          /* internal consistency check failed on the device */
#define RIDFA_E_TOO_LARGE (-12)      /* tables + scratch exceed RIDFA_NOALLOC_SCRATCH_BYTES */

#define RIDFA_UNDEF 0xFFFFu          /* chunk-map entry of a dead run */
#define RIDFA_MAX_STATES 65534u
#define RIDFA_MAX_SLOTS 256u         /* interface slots the device kernels support */
#define RIDFA_NOALLOC_SCRATCH_BYTES (4u << 20) /* fixed device array of ridfa_recognize_noalloc */

typedef struct ridfa_program ridfa_program;

typedef struct {
    uint32_t minimize_interface; /* 1: Nerode delegation, if_min (Sec. 3.4); 0: I^B = all singletons */
    uint32_t build_dfa;          /* 1: also build the minimal DFA for the all-states comparator */
    uint32_t max_states;         /* cap on |P| and |Q_DFA|; 0 means RIDFA_MAX_STATES */
} ridfa_compile_opts;

typedef struct {
    uint32_t n_nfa;          /* |Q_N| = number of positions + 1 (q0) */
    uint32_t n_states;       /* |P|, states of the RI-DFA B (Sec. 3.1) */
    uint32_t k;              /* interface slots |I^{B_min}| (= n_nfa without minimisation) */
    uint32_t n_classes;      /* byte classes C (bytes read by exactly the same positions) */
    uint32_t n_dfa_states;   /* |Q| of the minimal DFA (0 if not built) */
    uint32_t q0_slot;        /* slot of {q0} */
    uint64_t table_bytes;    /* device bytes of the RID tables */
    uint64_t dfa_table_bytes;/* device bytes of the DFA tables (0 if not built) */
} ridfa_info;

typedef struct {
    uint32_t piece_len;       /* intra-chunk speculation when the text has too few chunks to fill
                                 the GPU: each chunk is cut into pieces of about this many bytes,
                                 every piece is run (one warp, lockstep) from every state of the
                                 automaton, and the piece functions are composed into the chunk's
                                 exact map row.
                                 0 auto (on when the chunks would keep few of the resident warps
                                 busy -- fewer than warps / (4 * (1 + ceil(P/32))) chunks -- the
                                 automaton has at most RIDFA_MAX_SLOTS states and the chunks are
                                 long enough; pieces of 256 bytes or more); 1 off;
                                 >= 64 that piece length, when the other conditions hold */
    uint32_t block_threads;   /* threads per block of the reach kernel: 0 auto, a multiple of 32
                                 up to 1024 (512 when k > 128) */
    uint32_t probe_interval;  /* bytes between convergence checks of the speculative runs: 0 auto */
    uint32_t grid_blocks;     /* reach-kernel blocks: 0 auto (one wave on all SMs) */
    uint32_t profile;         /* 1: record CUDA events around the reach and join launches on the
                                 call's stream (read them back with ridfa_last_timings) */
    uint32_t table_mode;      /* reach-kernel table layout: 0 auto; 1 compact (premultiplied
                                 16-bit offsets in shared memory, else the uint16 table through
                                 generic loads); 2 lane-replicated 16-bit offsets; 3
                                 lane-replicated 32-bit offsets; 4 half-replicated (16 copies of
                                 the transition table); 5 the uint16 table through generic loads;
                                 6 lane-replicated 16-bit entries in 4-byte units (tables up to
                                 4x larger than mode 2 allows); 7 as 6 with one 512-byte copy of
                                 the class table (32 KB more for staging; text paths 1 and 5
                                 only); 8 two-byte steps: lane-replicated 16-bit entries for every
                                 pair of classes beside the single classes, so the converged runs
                                 take one transition lookup per two bytes (small automata:
                                 (P/2 + 1) * (C*C + C) <= 511; text paths 1 and 3 only); 9
                                 two-byte steps in one compact table of premultiplied 16-bit
                                 offsets (pair and single columns), a lane's runs sharing each
                                 pair's column ((P + 1) * (C*C + C) <= 32767; text paths 1 and 5
                                 only); 10 two-byte steps in F lane copies (the layout of 8 with
                                 16, 8, 4 or 2 copies side by side and rows of an odd number of
                                 words, at most 32/F wavefronts a lookup; F the most copies whose
                                 16-bit byte offsets fit and that leave shared memory for the
                                 launch's warps: (P/2 + 1) * ((C*C + C) | 1) * 4F <= 65535); 11 as
                                 10 with half-word offsets (twice the copies in 16 bits) and one
                                 256-byte table of 8-bit class offsets ((P/2 + 1) * ((C*C + C) | 1)
                                 * 2F <= 65535, (C - 1) * 2F <= 255); 10 and 11: text paths 1 and
                                 3 only (E_ARG if the chosen layout does not fit) */
    uint32_t text_path;       /* how the converged runs read the text: 0 auto; 1 each lane's own
                                 16-byte global loads; 2 retired (per-lane bulk copies; E_ARG);
                                 3 warp-cooperative coalesced loads staged in shared memory; 4
                                 the same with two chunks per lane, interleaved; 5 as 3, and a
                                 lane finishes all the runs its chunk handed off in one pass over
                                 the chunk (at most 512 threads a block).  3 to 5 need a
                                 16-byte-aligned d_text (E_ARG otherwise) */
    uint32_t lookback_cap;    /* pieces of automata with more than 256 states and k <= 32 start
                                 from look-back start sets of at most this many states (0 = 32,
                                 the largest; 1..32); a piece whose set stays larger has its whole
                                 function computed from every state instead.  E_ARG above 32 */
} ridfa_tuning;

/* Compile `re` (re_len bytes, need not be NUL-terminated) on the host: position NFA, RI-DFA
 * (incremental powerset N(q0) u N(q1) u ..., Sec. 3.1), Nerode partition and delegation
 * (Sec. 3.4), byte classes, uint16 transition tables; optionally the minimal DFA.  Device tables
 * are uploaded on first use by a recognize call (so this works without a GPU).
 * opts may be NULL (minimize_interface = 1, build_dfa = 1, max_states = 65534).  Every table
 * index the kernels compute unchecked is verified on the host before the program is returned.
 * Errors: E_ARG, E_SYNTAX, E_TOO_MANY_STATES, E_NOMEM, E_STATE (a table failed that check: an
 * internal error).  *out is set only on success. */
int ridfa_compile(const char *re, size_t re_len, const ridfa_compile_opts *opts,
                  ridfa_program **out);

/* Release a program, its host tables and (on every device it was uploaded to) its device
 * tables and scratch.  NULL is a no-op.  Must not race with calls using the program. */
void ridfa_free(ridfa_program *prog);

/* Sizes of the compiled automata.  Errors: E_ARG. */
int ridfa_program_info(const ridfa_program *prog, ridfa_info *out);

/* NFA states (0 = q0, p >= 1 = position p) contained in RI-DFA state `state` (the subset it
 * stands for, Sec. 3.1), ascending, into out[0..cap).  *n_out = subset size.
 * Errors: E_ARG (bad state or cap too small; *n_out still set). */
int ridfa_state_set(const ridfa_program *prog, uint32_t state, uint32_t *out, uint32_t cap,
                    uint32_t *n_out);

/* out[a] = representative NFA state of interface slot a (a < k), ascending (Sec. 3.4: the
 * lowest state of each language-equivalence class of singletons).  Errors: E_ARG. */
int ridfa_slots(const ridfa_program *prog, uint32_t *out);

/* out[q] = slot of the representative that NFA state q delegates to (q < n_nfa); this is the
 * interface function if_min on singletons (Sec. 3.4).  Errors: E_ARG. */
int ridfa_delegates(const ridfa_program *prog, uint32_t *out);

/* Host copies of the tables the device kernels use.  which = 0: RI-DFA, 1: minimal DFA.
 * trans: uint16 [(n+1) * n_classes] next state (row n and undefined moves = n, the dead
 * state); classmap: uint8 [256]; final: uint8 [n] (1 = in F^RID / F).  Any pointer may be
 * NULL.  Errors: E_ARG, E_NO_DFA. */
int ridfa_export_tables(const ridfa_program *prog, int which, uint16_t *trans,
                        uint8_t *classmap, uint8_t *final_flags);

/* ---- Sharded recognition (one text split into contiguous shards, e.g. one per GPU).
 * The join (Sec. 3.2) composes chunk relations associatively, so a shard -- a run of whole
 * chunks -- reduces to one relation: entered through interface slot a, its chunks lead to a set
 * of states at its end.  ridfa_recognize_shard computes that summary on the device (reach +
 * join over the shard's chunks); ridfa_join_shards composes the summaries of consecutive shards
 * on the host, entering shard j+1 through if_min of the states shard j ends in, and tests the
 * final set against F^RID.  Only the summaries (a few KB each) cross between shards. */
typedef struct {
    uint32_t k;                                   /* interface slots of the program */
    uint32_t n_out;                               /* distinct states the shard's last chunk ends in */
    uint16_t entry[RIDFA_MAX_SLOTS];              /* state after the shard's first chunk from slot a
                                                     (RIDFA_UNDEF: the run dies) */
    uint16_t out_state[RIDFA_MAX_SLOTS];          /* those end states, ascending */
    uint32_t reach[RIDFA_MAX_SLOTS][RIDFA_MAX_SLOTS / 32]; /* bit y of row a: entering through slot
                                                     a can end in out_state[y] */
} ridfa_shard_summary;

/* Summary of the shard d_text[0, len) cut into n_chunks chunks (1 <= n_chunks <= len), written
 * to the host struct *h_out; synchronises `stream`.  Errors: as ridfa_recognize. */
int ridfa_recognize_shard(const ridfa_program *prog, const uint8_t *d_text, size_t len, uint32_t n_chunks,
                          const ridfa_tuning *tuning, ridfa_shard_summary *h_out, void *stream);

/* Accept bit of the text made of n_shards consecutive shards (the first one starts the text),
 * from their summaries; host only.  Errors: E_ARG (NULL, n_shards == 0, a summary of another
 * program's k). */
int ridfa_join_shards(const ridfa_program *prog, const ridfa_shard_summary *shards, uint32_t n_shards,
                      uint8_t *h_accept);

/* Per-chunk join states (the join of Sec. 3.2 as a full scan instead of a reduction), from the
 * chunk maps of one recognition of `prog` (d_maps: device [n_chunks][k], as written by
 * ridfa_recognize with d_chunk_maps).  d_entry (device, uint32 [n_chunks][ceil(k/32)], or NULL)
 * receives, per chunk i, the bit set E_i = if_min(PLAS_{i-1}) ∩ PIS_i of interface slots the
 * chunk is entered through (E_1 = {q0's slot} ∩ PIS_1), so that PLAS_i = λ_i(E_i); *h_reject
 * is the first chunk (0-based) whose PLAS_i is empty -- where the text is rejected -- or -1.
 * Synchronises `stream`.  Errors: E_ARG, E_UNSUPPORTED, E_NOMEM, E_CUDA, E_STATE. */
int ridfa_join_scan(const ridfa_program *prog, const uint16_t *d_maps, uint32_t n_chunks, uint32_t *d_entry,
                    int64_t *h_reject, void *stream);

/* Transition counts of the reach phase, computed on the host (diagnostics).
 * Chunk 1 runs from {q0}'s slot only, every other chunk from every interface slot (Sec. 3.2);
 * which = 1 counts the all-states DFA comparator instead (chunk 1 from q0, the others from
 * every state of the minimal DFA, Sec. 2); which = 2 the NFA variant (chunk 1 from q0, the others
 * from every position-NFA state, each start's set of active states followed on its own: a step
 * from the set S on a byte of class c executes sum over q in S of |Follow(q) n positions(c)|
 * transitions, counted in w_paper; w_conv then counts the active NFA states processed). */
typedef struct {
    uint64_t w_paper;   /* transitions with every run followed on its own, undefined moves not
                           counted: the paper's measure (Sec. 1, Fig. 1) */
    uint64_t w_conv;    /* table lookups when runs in the same state at the same position are
                           merged: distinct live states summed over positions */
    uint64_t runs;      /* runs started: 1 + (n_chunks - 1) * k */
    uint64_t dead_runs; /* runs that met the undefined move before their chunk end */
    uint64_t converge_hist[16]; /* chunks 2..c by the bytes read until their runs leave at most
                           one live state (convergence, Sec. 5; merged runs, dead runs dropped):
                           bucket 0 for 0 or 1 byte, bucket b for 2^b .. 2^(b+1) - 1 bytes
                           (b <= 14), bucket 15 for chunks still holding two or more live states
                           at their end.  Zero for which = 2. */
} ridfa_transition_counts;

/* h_text: host pointer to len bytes; 1 <= n_chunks <= len; n_threads host threads over the
 * chunks (0 = all hardware threads).  Errors: E_ARG, E_NO_DFA, E_UNSUPPORTED (which = 2 with more
 * than 128 NFA states), E_CHUNKS, E_NOMEM. */
int ridfa_count_transitions(const ridfa_program *prog, int which, const uint8_t *h_text, size_t len,
                            uint32_t n_chunks, uint32_t n_threads, ridfa_transition_counts *out);

/* The same recognition on the host's cores, the CPU context of the device numbers (the paper
 * measures its method on the cores of one machine, Sec. 4).  n_chunks = 1: the serial recognizer,
 * the table loop from {q0} (Sec. 2; which = 1: the classic serial run of the minimal DFA).
 * n_chunks > 1: the chunked speculative recognition of Sec. 3.2 -- chunk 1 from {q0}'s slot, every
 * other chunk from every interface slot, runs that meet in one state at one position merged, then
 * the join PLAS_i = lambda_i(if_min(PLAS_{i-1})) and PLAS_c n F^RID != {} -- with the chunks split
 * over n_threads host threads (0 = all hardware threads) and the join on the calling thread;
 * which = 1: the all-states DFA variant (Sec. 2).  Chunk boundaries as on the device.  h_text:
 * host pointer to len bytes; len == 0 needs n_chunks == 0 (the answer is whether the empty word
 * is in L).  *h_accept = 1 if text in L(RE) else 0.  ridfa_recognize never calls this (no host
 * fallback exists); it holds c * k uint16 chunk maps in host memory while it runs.
 * Errors: E_ARG, E_NO_DFA, E_CHUNKS, E_NOMEM. */
int ridfa_cpu_recognize(const ridfa_program *prog, int which, const uint8_t *h_text, size_t len,
                        uint32_t n_chunks, uint32_t n_threads, uint8_t *h_accept);

/* Recognize one text resident on the device (the RID: reach + join, Sec. 3.2).
 * d_text: device pointer to len bytes (any alignment).  n_chunks: c, 1 <= c <= len.
 * len == 0 is allowed with n_chunks == 0: the answer is whether the empty word is in L.
 * tuning: NULL = automatic.  *h_accept = 1 if text in L(RE) else 0.  d_chunk_maps: NULL, or a
 * device buffer of n_chunks * k uint16 that receives the chunk maps lambda_i.
 * Synchronises `stream` before returning.
 * Errors: E_ARG, E_CHUNKS, E_UNSUPPORTED (k > RIDFA_MAX_SLOTS), E_NOMEM, E_CUDA, E_STATE. */
int ridfa_recognize(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                    uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *h_accept,
                    uint16_t *d_chunk_maps, void *stream);

/* Failure detection of device waits: the library's bounded mbarrier wait (at most a fixed number
 * of polls, then E_TIMEOUT with the context intact; the form any spin on a flag or barrier in
 * these kernels must take -- the recognize kernels themselves currently have none, their tickets
 * being atomics), exercised alone on `stream`.  One warp waits for the first phase of a fresh mbarrier, at most `limit` polls; with
 * arrive != 0 the phase is completed first (returns RIDFA_OK), with arrive == 0 nothing arrives and
 * the call returns RIDFA_E_TIMEOUT.  Allocates 4 device bytes; synchronises `stream`.
 * Errors: E_NOMEM, E_CUDA. */
int ridfa_check_bounded_wait(uint32_t limit, int arrive, void *stream);

/* Recognize one text held in host memory: the len bytes at h_text are copied to the caller's
 * device buffer d_staging (at least len bytes; 16-byte aligned for the staged text paths) on
 * `stream`, then recognized as by ridfa_recognize; the accept bit comes back in *h_accept.
 * h_text may be page-locked (a direct copy at the link's rate) or pageable (staged by the
 * driver).  Ownership: both buffers stay the caller's; d_staging holds the text afterwards.
 * Synchronises `stream`.  Errors: as ridfa_recognize; E_ARG also for a null h_text or d_staging
 * with len > 0. */
int ridfa_recognize_host(const ridfa_program *prog, const uint8_t *h_text, size_t len,
                         uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_staging,
                         uint8_t *h_accept, void *stream);

/* As ridfa_recognize, but the accept byte goes to device memory d_accept (1 byte) and nothing
 * is synchronised: the result is valid once `stream` reaches this point.  Device status
 * (E_STATE) is then reported by the next call on the program, or by ridfa_last_status(). */
int ridfa_recognize_async(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                          uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_accept,
                          uint16_t *d_chunk_maps, void *stream);

/* The all-states DFA comparator (the DFA variant of the classic algorithm, Sec. 2): every
 * state of the minimal DFA is speculated on; chunk maps are [n_chunks][n_dfa_states].
 * Same arguments and errors as ridfa_recognize, plus E_NO_DFA. */
int ridfa_recognize_dfa(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                        uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *h_accept,
                        uint16_t *d_chunk_maps, void *stream);

int ridfa_recognize_dfa_async(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                              uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_accept,
                              uint16_t *d_chunk_maps, void *stream);

/* The NFA variant of the classic algorithm (Sec. 2; the NFA columns of Table 3), a comparator
 * for the RID.  The chunk automaton is the position NFA with every state initial (chunk 1: q0
 * only); each start state q's set of active states is simulated over the chunk on its own, with no
 * merging of runs, giving lambda_i(q) = rho(q, y_i), the set of NFA states reached (empty: q is
 * not in PIS_i).  The join composes the chunk relations, PLAS_i = lambda_i(PLAS_{i-1}), as a tree
 * of relation compositions on the device; the text is accepted iff PLAS_c meets F.
 *   d_text: device pointer to len bytes; n_chunks: 1 <= c <= len (len == 0 needs c == 0).
 *   d_sets: NULL, or a device buffer of n_chunks * n_nfa * ceil(n_nfa / 32) uint32 receiving the
 *   rows lambda_i(q) (row (i, q) at word (i * n_nfa + q) * ceil(n_nfa / 32); bit p of its word
 *   p / 32 = NFA state p, 0 = q0, p >= 1 = position p); chunk 1 fills only q0's row.
 *   *h_accept = 1 if the text is in L(RE).  Synchronises `stream`.  The library allocates (and
 * keeps, per program and device) scratch of about n_chunks * n_nfa * ceil(n_nfa / 32) * 4 bytes
 * when d_sets is NULL.
 * Errors: E_ARG, E_CHUNKS, E_UNSUPPORTED (more than 128 NFA states), E_NOMEM, E_CUDA. */
int ridfa_recognize_nfa(const ridfa_program *prog, const uint8_t *d_text, size_t len, uint32_t n_chunks,
                        uint8_t *h_accept, uint32_t *d_sets, void *stream);

/* The paper has no counterpart to this call.  It is the RID path (the same reach and join
 * kernels as ridfa_recognize_async) for callers that must not allocate device memory while they
 * run: cudaMalloc can stall every stream of the device and can fail when another framework's
 * caching allocator already holds the memory, so latency-bound services, and plug-ins whose host
 * application owns all device allocations, need a recognize call that allocates nothing.
 * No cudaMalloc, cudaFree or other allocating routine is called.  The program's tables and all
 * kernel scratch live in one fixed device array of RIDFA_NOALLOC_SCRATCH_BYTES (4 MiB) that
 * every GPU loading the library holds until the process exits.
 *   d_text: device pointer to len bytes; n_chunks: 1 <= c <= len (len == 0 needs c == 0).
 *   d_accept: device byte, receives 1 if the text is in L(RE) else 0 (written on `stream`).
 *   d_chunk_maps: REQUIRED device buffer of n_chunks * k uint16 (the chunk maps, as in
 *   ridfa_recognize).  Nothing is synchronised.
 * Limits: the tables plus 4 bytes per chunk plus about 133 KiB of join scratch must fit in the
 * array, otherwise RIDFA_E_TOO_LARGE and nothing is launched.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process, so the library must not be used across a
 * cudaDeviceReset of that device.  The
 * device status word (the join's consistency check, E_STATE on ridfa_recognize) is not reported
 * by this call, which returns once its work is queued.  Every call copies the program's tables into
 * the array and clears the counters the join needs; the array keeps the last call's contents.
 * Calls that overlap on the GPU (on different streams, from different threads or programs) use
 * the same array and race: serialise them.
 * Errors: E_ARG, E_CHUNKS, E_UNSUPPORTED (k > RIDFA_MAX_SLOTS), E_TOO_LARGE, E_CUDA. */
int ridfa_recognize_noalloc(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                            uint32_t n_chunks, uint8_t *d_accept, uint16_t *d_chunk_maps,
                            void *stream);

/* Synchronise `stream` and report the device status word of the program's last call
 * (RIDFA_OK or E_STATE).  Errors: E_ARG, E_CUDA. */
int ridfa_last_status(const ridfa_program *prog, void *stream);

/* Device time of the last profiled call's reach kernel and join kernel, in milliseconds,
 * from CUDA events recorded on that call's stream (tuning->profile = 1).  Waits for the
 * events.  Errors: E_ARG (no profiled call yet), E_CUDA. */
int ridfa_last_timings(const ridfa_program *prog, float *reach_ms, float *join_ms);

/* The reach plan of the last ridfa_recognize / ridfa_recognize_dfa / ridfa_recognize_host call of
 * `prog` on the current device (diagnostics; the automatic choices the tuning fields override). */
typedef struct {
    uint32_t table_mode;    /* table layout, numbered as ridfa_tuning::table_mode (1..11) */
    uint32_t text_path;     /* 1 global loads, 3 staged, 4 staged two chunks a lane, 5 set path */
    uint32_t lane_copies;   /* copies F of layouts 10 and 11, else 0 */
    uint32_t block_threads; /* threads per block of the reach launch */
    uint32_t grid_blocks;   /* blocks of the reach launch */
    uint32_t pieces;        /* 1: the chunks were cut into pieces (intra-chunk speculation) */
} ridfa_plan_report;
/* Errors: E_ARG (prog or out NULL, or no call on this device yet), E_CUDA. */
int ridfa_last_plan(const ridfa_program *prog, ridfa_plan_report *out);

/* ---- Batched recognition (the paper recognises one text at a time; a batch runs the same
 * reach and join, exactly, for many (text, program) items at once).
 * All items' chunks run in one persistent reach launch per shared-memory table layout (CTAs take
 * tasks of up to 32 chunks per warp of one program from an atomic ticket and reload their tables
 * only when the program changes) followed by one join launch over all texts; create() captures
 * these launches into a CUDA graph that run() replays. */
typedef struct {
    const uint8_t *d_text;   /* device pointer (16-byte alignment of every text enables the
                                cooperative staged text path; otherwise global loads are used) */
    uint64_t len;            /* bytes; 0 allowed (accept = empty word in L) */
    uint32_t prog;           /* index into progs[] */
    uint32_t n_chunks;       /* 0: ceil(len / chunk_len); else 1 <= n_chunks <= len */
} ridfa_batch_item;

typedef struct {
    uint32_t chunk_len;      /* bytes per chunk for items with n_chunks == 0; 0 = autotune: chunk
                                length and launch shape are looked up in a cache keyed by every
                                program's (log2 |P|, log2 k, log2 C), else timed on this batch --
                                chunk lengths 4-32 KiB, then warps per block (all that fit, 16,
                                8), then the run interleave below -- and the winner is cached
                                under those keys */
    uint32_t no_graph;       /* 1: run() enqueues the launches directly instead of a CUDA graph */
    uint32_t block_warps;    /* warps per block of the reach launches at most (threads per task
                                group); 0 = as many as fit (tuned when chunk_len == 0); <= 32 */
    uint32_t set_mode;       /* tables too large to replicate (runs that stay apart): 1 a lane
                                carries all of its chunk's runs, interleaved, through one pass; 2
                                one run per lane; 0 = 1 (tuned when chunk_len == 0) */
} ridfa_batch_opts;

typedef struct {
    uint64_t total_bytes;
    uint64_t total_chunks;
    uint32_t n_programs, n_launches, n_tasks, n_segments;
    uint32_t chunk_len;      /* the chunk length in use */
    uint32_t block_warps;    /* warps per block cap in use (0: as many as fit) */
    uint32_t set_mode;       /* run interleave in use (0/1 set path, 2 one run per lane) */
    uint32_t graph;          /* 1 if run() launches a CUDA graph */
    uint64_t device_bytes;   /* device memory the batch holds (descriptors, maps, summaries) */
} ridfa_batch_stats;

typedef struct ridfa_batch ridfa_batch;

/* Plan a batch: per-program device tables (uploaded if needed), chunking, tasks, join segments,
 * device scratch (one allocation), and the CUDA graph.  The texts and d_accept (n_items bytes,
 * device; d_accept[i] receives item i's accept bit) must stay valid while the batch is used; the
 * programs must outlive it.  Errors: E_ARG, E_CHUNKS, E_UNSUPPORTED, E_NOMEM, E_CUDA. */
int ridfa_batch_create(const ridfa_program *const *progs, uint32_t n_progs,
                       const ridfa_batch_item *items, uint32_t n_items, uint8_t *d_accept,
                       const ridfa_batch_opts *opts, ridfa_batch **out);

/* Enqueue the whole batch on `stream` (one graph launch); asynchronous.  Runs of one batch must
 * not overlap.  Errors: E_ARG, E_CUDA. */
int ridfa_batch_run(ridfa_batch *batch, void *stream);

int ridfa_batch_get_stats(const ridfa_batch *batch, ridfa_batch_stats *out);

/* Synchronise the batch's device and release it.  NULL is a no-op. */
void ridfa_batch_free(ridfa_batch *batch);

/* One-shot: create (chunk length 8 KiB, no graph), run on `stream`, synchronise, free. */
int ridfa_recognize_batch(const ridfa_program *const *progs, uint32_t n_progs,
                          const ridfa_batch_item *items, uint32_t n_items, uint8_t *d_accept,
                          void *stream);

/* ---- Served recognition (the paper has no serving layer; each request is recognised exactly
 * as ridfa_recognize would, reach + join of Sec. 3.2).
 * A server keeps programs resident and owns one CUDA device: a text arena in device memory with
 * a pinned host mirror, and n_streams launch slots, each with its own stream, descriptor image
 * and scratch.  ridfa_server_submit() admits a request (copying a host text into the arena's
 * mirror) or refuses it with E_BUSY; a scheduler thread forms a batch from every request pending
 * whenever a launch slot is free (continuous batching: requests that arrive while batches run
 * join the next one), copies the batch's texts to the device, runs the batched reach and join
 * on that slot's stream and posts one result per request; ridfa_server_poll() collects them. */
typedef struct {
    int32_t device;             /* CUDA device ordinal (-1: the current device) */
    uint32_t n_streams;         /* launch slots (batches in flight); 0 = 3 */
    uint64_t arena_bytes;       /* device text arena (and its pinned mirror); 0 = 1 GiB */
    uint32_t max_requests;      /* requests admitted and not yet polled; 0 = 1 << 20 */
    uint32_t max_batch_requests;/* requests per batch; 0 = 8192 */
    uint64_t max_batch_bytes;   /* text bytes per batch; 0 = 512 MiB */
    uint32_t chunk_len;         /* bytes per chunk; 0 = adapted per batch: about two chunks per
                                   resident lane of the GPU, a power of two in [1 KiB, 8 KiB] */
    uint32_t reserved;
    uint64_t device_budget;     /* admission by device memory: the resident programs' tables plus,
                                   for every admitted and unfinished request, its arena text and
                                   its kernel scratch (chunk maps and summaries, 2k + 4 bytes per
                                   chunk of at least chunk_len -- 1 KiB when adaptive -- plus 64)
                                   may not exceed this many bytes; 0 = no budget (the arena and
                                   max_requests alone admit) */
} ridfa_server_opts;

typedef struct {
    uint64_t req_id;
    int32_t status;             /* RIDFA_OK, or RIDFA_E_STATE / RIDFA_E_CUDA for this request */
    uint32_t accept;            /* 1 if the text is in L(RE) */
    double latency_us;          /* submit to result posted, host steady clock */
} ridfa_result;

typedef struct {
    uint64_t submitted, completed, rejected, batches, bytes;
    uint32_t max_batch, n_programs;
    uint64_t device_bytes;      /* arena + slot scratch */
    uint64_t table_bytes;       /* device tables of the resident programs (charged to the budget) */
    uint64_t budget_used;       /* tables + admitted unfinished requests, now */
    uint64_t budget_peak;       /* ... and its largest value so far */
    uint32_t batch_hist[16];    /* batches by size: bucket b counts batches of 2^b .. 2^(b+1)-1
                                   requests (the last bucket: 2^15 and more) */
} ridfa_server_stats;

typedef struct ridfa_server ridfa_server;

#define RIDFA_SUBMIT_DEVICE_TEXT 1u /* submit flag: `text` is a device pointer, used in place; it
                                       must stay valid until the request's result is polled */

/* Create a server (opts may be NULL) and start its scheduler thread.
 * Errors: E_ARG, E_NOMEM, E_CUDA. */
int ridfa_server_create(const ridfa_server_opts *opts, ridfa_server **out);

/* Make `prog` resident (tables uploaded now) and return its slot for submit().  The program
 * must outlive the server.  With a device_budget its table bytes (ridfa_info.table_bytes) are
 * charged to the budget for the server's life; E_BUSY when they do not fit beside what is
 * already charged (nothing is added then).
 * Errors: E_ARG, E_UNSUPPORTED (k > RIDFA_MAX_SLOTS), E_BUSY, E_NOMEM, E_CUDA. */
int ridfa_server_add_program(ridfa_server *srv, const ridfa_program *prog, uint32_t *prog_slot);

/* Submit one request: recognise text[0, len) with program `prog_slot`.  A host text is copied
 * before the call returns; a device text (RIDFA_SUBMIT_DEVICE_TEXT) is read in place.
 * Admission: the arena must have room for a host text, fewer than max_requests may be
 * outstanding, and with a device_budget the request's charge (its arena text, none for a device
 * text, plus its scratch) must fit beside the tables and the requests still unfinished; the
 * charge is released when the result is posted.
 * Errors: E_ARG, E_BUSY (arena, request count or device budget full: poll, then retry),
 * E_TOO_LARGE (the text alone exceeds the arena or a batch, or its charge exceeds the budget
 * left beside the tables). */
int ridfa_server_submit(ridfa_server *srv, uint32_t prog_slot, const uint8_t *text, uint64_t len,
                        uint32_t flags, uint64_t *req_id);

/* Move up to max finished results to out (*n_out of them), waiting up to wait_us microseconds
 * for the first one.  Errors: E_ARG. */
int ridfa_server_poll(ridfa_server *srv, ridfa_result *out, uint32_t max, uint32_t *n_out, uint32_t wait_us);

/* Wait until every submitted request has finished (results may still be unpolled), at most
 * timeout_ms milliseconds.  Errors: E_ARG, E_TIMEOUT. */
int ridfa_server_drain(ridfa_server *srv, uint32_t timeout_ms);

int ridfa_server_get_stats(const ridfa_server *srv, ridfa_server_stats *out);

/* Stop the scheduler, wait for work in flight and release everything.  NULL is a no-op. */
void ridfa_server_destroy(ridfa_server *srv);

/* Open-loop Poisson load generator for a server (a measurement client; the paper has no
 * counterpart).  Arrivals at rate_rps for `seconds` (exponential gaps, seeded); each arrival
 * submits a uniformly chosen text of the caller's pool with its program slot and submit_flags
 * (0: host texts, copied into the arena; RIDFA_SUBMIT_DEVICE_TEXT: device texts, read in place,
 * so that the client's copies do not limit the rate), retrying while the server answers E_BUSY,
 * and polls results in between.
 * Latency of a request = (submit time - scheduled arrival) + the server's submit-to-result time,
 * so a client or server that falls behind is charged for it.  Runs on the calling thread and
 * returns when every request's result has been polled.
 *   prog_slots[i], texts[i], lens[i]: the pool (n_texts entries); records: out[0..cap), one per
 *   request in arrival order (*n_out of them); *wall_s: seconds from the first arrival to the
 *   last result.
 * Errors: E_ARG (bad arguments, or more arrivals than cap), E_TOO_LARGE, errors of submit. */
typedef struct {
    uint32_t text;              /* pool index of the request's text */
    int32_t status;             /* the request's result status */
    uint32_t accept;            /* 1 if accepted */
    uint32_t busy_retries;      /* submits refused with E_BUSY before this one was admitted */
    double latency_us;          /* scheduled arrival to result posted */
    double server_us;           /* submit to result posted (the server's own measure) */
} ridfa_loadgen_record;

int ridfa_bench_served_poisson(ridfa_server *srv, const uint32_t *prog_slots,
                               const uint8_t *const *texts, const uint64_t *lens, uint32_t n_texts,
                               double rate_rps, double seconds, uint64_t seed,
                               ridfa_loadgen_record *out, uint32_t cap, uint32_t *n_out,
                               double *wall_s, uint32_t submit_flags);

/* Roofline microbenchmarks (diagnostics; the paper has no counterpart).  Both allocate a 4-byte
 * sink and synchronise the current device.
 * ridfa_bench_smem_gather: the reach kernel's converged step alone -- per text byte one
 *   lane-private shared-memory gather for the byte's class and one for the next state (dependent
 *   on the previous state) -- on every SM with 1024 threads, `iters` bytes per thread.  Returns
 *   the rate in text bytes per second (*ms_out: the timed launch).  Errors: E_ARG, E_CUDA.
 * ridfa_bench_hbm_read: streaming read of `bytes` of a 16-byte-aligned device buffer with 16-byte
 *   loads; returns bytes per second.  Errors: E_ARG, E_CUDA. */
int ridfa_bench_smem_gather(uint32_t iters, double *bytes_per_s, double *ms_out);
int ridfa_bench_hbm_read(const uint8_t *d_buf, size_t bytes, double *bytes_per_s, double *ms_out);

/* Static text of a status code. */
const char *ridfa_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* RIDFA_H */
