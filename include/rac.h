/*
 * rac.h -- C ABI of the B300 arc-consistency library (librac.so).
 *
 * The library enforces arc consistency on binary constraint networks with
 * the recurrent formulation of "Paralleling and Accelerating Arc Consistency
 * Enforcement with Recurrent Tensor Computations" (arXiv 2407.11388):
 *
 *   Eq. 1 (Sec. 3):  Dt^(0) = {},
 *                    Dt^(k) = Dt^(k-1) U {(x,a) | exists y: c_xy|_(x,a) is a
 *                                          subset of Dt^(k-1)},
 *
 * swept synchronously until a sweep removes nothing; the result D \ Dt^(K) is
 * D_ac, the union of every arc-consistent subset of D (Sec. 3, Prop. 1).  In
 * tensor form (Sec. 4, Fig. 1, Algorithm 1 `tensorRevise`) each sweep counts
 * Sup_xy[a] = sum_b R_xy[a][b] * D[y][b] for every value (x,a) and every
 * constraint c_xy on x, and keeps (x,a) only if every count is non-zero.
 *
 * Conventions shared by every entry point:
 *  - A network has n_vars variables, all with values 0..d-1, 1 <= d <= 32.
 *  - A domain state is n_vars uint32 words; bit a of word x is set iff value
 *    a is in dom(x).  Bits >= d must be zero.
 *  - Supports are taken inside the domain passed in (the paper's listing
 *    multiplies the constraint tensor by the domain mask, Appendix E): a
 *    value with no allowed partner left in the neighbour's domain is removed.
 *  - `iterations` counts every sweep executed, including the last sweep,
 *    which removes nothing (the loop trips of Algorithm 1).  A domain that is
 *    already arc consistent takes 1 sweep.
 *  - Per-state results: status RAC_OK (fixpoint, no empty domain),
 *    RAC_WIPEOUT (some domain of the result is empty), RAC_ETIMEOUT (the
 *    sweep cap was reached first) or RAC_EBARRIER (a device-side wait gave
 *    up after its time limit; the domains are then unspecified, and the
 *    scratch workspace of that (network, stream) is poisoned: every later
 *    call on it reports RAC_EBARRIER without enforcing).
 *  - Functions return RAC_OK or a negative error code; on error nothing has
 *    been launched and rac_last_error() describes the cause.  No C++
 *    exception crosses this boundary: a host allocation that fails inside
 *    the library is RAC_ENOMEM, any other host-side exception RAC_EINVAL.
 *  - Device pointers are plain CUDA device addresses (for example the
 *    data_ptr() of a torch tensor on the same device).  `stream` is a
 *    cudaStream_t; NULL means the legacy default stream.  Work is enqueued on
 *    `stream` and the call returns without waiting unless stated otherwise.
 */
#ifndef RAC_H
#define RAC_H

#include <stdint.h>

#if defined(__GNUC__)
#define RAC_API __attribute__((visibility("default")))
#else
#define RAC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rac_network rac_network;
typedef struct CUstream_st *rac_stream_t; /* same type as cudaStream_t */
typedef int32_t rac_status;

/* Return and per-state status codes. */
#define RAC_OK 0
#define RAC_WIPEOUT 1
#define RAC_EINVAL (-1)
#define RAC_ENOMEM (-2)
#define RAC_ECUDA (-3)
#define RAC_ETIMEOUT (-4)
#define RAC_EBARRIER (-5)
#define RAC_ENOTSUP (-6)

/* layout_flags of rac_create_network */
#define RAC_LAYOUT_BITS 0x1u /* bit-packed relation slabs (always built) */
/* The tensor-core kernel's operand store (RAC_KERNEL_TENSOR), built on the
 * device at creation: every relation in both orientations (its rows R[a][.]
 * and its columns R[.][b]), a 32-bit word per row or column, grouped by
 * 32 x 32-variable tile in the order the kernel's MMAs consume them, plus
 * each tile's presence rows: 256 KiB per tile that holds a constraint (138
 * MB for n = 1000, 528 MB for n = 2000).  The kernel expands each word to the
 * MMA's FP8 (E5M2) operand in tensor memory as it goes.  Without it the
 * first RAC_KERNEL_TENSOR call on the network builds it (an allocation and a
 * wait on its stream). */
#define RAC_LAYOUT_FP8 0x2u
/* Packed relation rows: row a of a relation takes bits [w a, w a + w) of the
 * relation's words, w = round_up(d, 4), instead of a word of its own, so a
 * relation takes ceil(w^2 / 32) words instead of w (d = 20: 13 words instead
 * of 20; d = 24: 18 instead of 24) and every sweep reads that much less.
 * Each row is shifted out of its word (or out of two, when it straddles
 * them) before the support test, one more instruction per row.  Every entry
 * point and kernel reads both layouts; the results and sweep counts do not
 * depend on it.  For d > 28 a row is a whole word already and the flag
 * changes nothing. */
#define RAC_LAYOUT_PACKED 0x4u
/* Rows of the relation tiles ("slabs": 32 column variables x `rows` row
 * variables of one block pair, read as one unit): RAC_LAYOUT_ROWS(l) asks
 * for 2^l rows, 1 <= l <= 5 (a tile's header of 2 x rows words keeps the
 * relations and the tile 16-byte aligned only from 2 rows on); without it the
 * largest power of two whose slab fits the kernels' 32 KiB staging buffer
 * (rows x 32 x 4 bytes x the words of a relation) is used.  The result and
 * the sweep count do not depend on it. */
#define RAC_LAYOUT_ROWS(l) ((uint32_t)((l) + 1) << 8)
#define RAC_LAYOUT_ROWS_MASK 0xF00u
/* CTAs of the network's persistent launches (the bit-packed kernel):
 * RAC_LAYOUT_MAX_CTAS(c), 1 <= c <= 65535, caps the grid at c.  Without it
 * the grid is every resident CTA of the GPU, capped at the number of tiles:
 * CTA c owns tiles c, c + G, ..., so a CTA beyond the tile count would only
 * take part in the sweep barriers.  The result and the sweep count do not
 * depend on it. */
#define RAC_LAYOUT_MAX_CTAS(c) ((uint32_t)(c) << 16)
#define RAC_LAYOUT_MAX_CTAS_MASK 0xFFFF0000u

/* flags of the enforce calls */
#define RAC_STOP_ON_WIPEOUT 0x1u /* end after the first sweep that leaves a domain
                                    empty and return that sweep's state
                                    (Algorithm 1 throws there; the listing of
                                    Appendix E returns None there).  Default: run
                                    Eq. 1 to its fixpoint. */
#define RAC_INCREMENTAL 0x2u     /* Proposition 2: sweep k >= 2 re-reads only
                                    the relation slabs touching a variable whose
                                    domain changed in sweep k-1.  The result,
                                    every sweep's removals and the sweep count
                                    are identical to the plain recurrence. */
#define RAC_VERIFY_FULL 0x4u      /* rac_enforce_learned only: the verification sweep
                                    after a gated sweep that removed nothing
                                    evaluates EVERY slab, instead of the slabs
                                    left pending (see rac_enforce_learned). */
#define RAC_KERNEL_TENSOR 0x10u  /* evaluate the support counts with the tensor-core
                                    kernel (tcgen05 FP8 MMAs: 128 relation rows x
                                    the running states x 32 values, FP32
                                    accumulation in tensor memory) instead of the
                                    bit-packed kernel:
                                    rac_enforce, single-network rac_enforce_batch
                                    and rac_enforce_host only, at most 128 states
                                    per launch (larger batches are split).  It
                                    reads the network's operand store
                                    (RAC_LAYOUT_FP8), which the first such call
                                    builds if the network has none: make that
                                    call outside any stream capture.  Results
                                    are identical. */
#define RAC_TEST_WITHHOLD_ARRIVAL 0x80000000u
                                 /* test hook for failure detection: one CTA
                                    withholds its first grid-barrier arrival,
                                    so every other CTA's bounded wait runs out
                                    (after 50 ms instead of 2 s); the call then
                                    reports RAC_EBARRIER for every state and
                                    poisons its workspace.  Nothing faults or
                                    hangs; not for production use. */

/*
 * rac_create_network -- copy a network into device memory in the library's
 * own layout.
 *
 *  n_vars     number of variables, 1 <= n_vars <= 2,000,000.
 *  d          domain size, 1 <= d <= 32.
 *  n_cons     number of constraints (>= 0).
 *  scope      HOST, n_cons x 2 int32: constraint c has scope (scope[2c],
 *             scope[2c+1]); both in [0, n_vars), different, and each
 *             unordered pair at most once (several relations on one pair
 *             would have to be intersected first).
 *  rel_bits   HOST, n_cons x d uint32: word a of constraint c has bit b set
 *             iff the pair (first variable = a, second variable = b) is
 *             allowed, i.e. R_xy[a][b] of the paper's relation tensor
 *             Cons[x][y][a][b] (Algorithm 2 `init`).  R_yx is R_xy
 *             transposed (one relation per scope, Sec. 2).  Bits >= d must be
 *             zero.  Variables with no constraint between them are
 *             unconstrained (only real constraints are in C_x).
 *  layout_flags  RAC_LAYOUT_BITS (0 means the same), optionally |
 *             RAC_LAYOUT_PACKED, RAC_LAYOUT_FP8, RAC_LAYOUT_ROWS(l),
 *             RAC_LAYOUT_MAX_CTAS(c); a tile too large for the staging
 *             buffer is rejected with RAC_EINVAL.
 *  out        receives the network handle.
 *
 * The library keeps its own copy; the host arrays may be freed on return.
 * The call synchronises with the device (allocation and upload).
 * Errors: RAC_EINVAL (bad argument, duplicate pair, bit >= d set, more
 * constraints than the n_vars (n_vars - 1) / 2 pairs), RAC_ENOMEM (host or
 * device allocation failed), RAC_ECUDA.
 */
RAC_API rac_status rac_create_network(int32_t n_vars, int32_t d, int64_t n_cons, const int32_t *scope,
                              const uint32_t *rel_bits, uint32_t layout_flags,
                              rac_network **out);

/*
 * rac_create_network_u8 -- rac_create_network from the relation tensor's 0/1
 * matrices instead of packed rows.
 *
 *  rel        HOST, n_cons x d x d uint8: rel[(c * d + a) * d + b] is
 *             R_xy[a][b] for (x, y) = (scope[2c], scope[2c+1]), 1 = the pair
 *             of values is allowed, 0 = it is not (the blocks of Algorithm 2's
 *             `init` relation tensor Cons[x][y][a][b], one per constraint).
 *
 * Row a of each matrix is packed on the host into the word rac_create_network
 * takes (bit b = R_xy[a][b]); the network, its layout and every result are
 * then those of rac_create_network on the packed words.  The other arguments,
 * ownership and errors are as there; an entry other than 0 or 1 is
 * RAC_EINVAL (the message names the constraint), checked before anything is
 * allocated on the device.
 */
RAC_API rac_status rac_create_network_u8(int32_t n_vars, int32_t d, int64_t n_cons,
                                         const int32_t *scope, const uint8_t *rel,
                                         uint32_t layout_flags, rac_network **out);

/* rac_destroy -- free a network and all device memory it owns (NULL-safe).
 * The caller must make sure no enforcement on it is still running. */
RAC_API void rac_destroy(rac_network *net);

/*
 * rac_enforce -- arc consistency for one domain state (Eq. 1 to its
 * fixpoint, one persistent kernel launch, no host round trip per sweep).
 *
 *  dom_in      DEVICE, n_vars words: the input domain D.
 *  dom_out     DEVICE, n_vars words: receives D_ac (or the state at which
 *              enforcement stopped).  dom_out == dom_in is allowed; any
 *              other overlap is not.
 *  iterations  DEVICE int32: sweeps executed.
 *  status      DEVICE int32: per-state status (see above).
 *  max_sweeps  sweep cap; <= 0 means none (Prop. 1 bounds the sweeps by
 *              |D| + 1 anyway).
 *  flags       RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL.
 *
 * Scratch memory comes from a per-(network, stream) workspace that the first
 * call on a stream allocates; calls on one stream reuse it, so capture such
 * calls in a CUDA graph only after one call on that stream has run.
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
RAC_API rac_status rac_enforce(const rac_network *net, const uint32_t *dom_in, uint32_t *dom_out,
                       int32_t *iterations, int32_t *status, int32_t max_sweeps, uint32_t flags,
                       rac_stream_t stream);

/*
 * rac_assign_enforce -- one step of backtrack search (Algorithm 2): `assign`
 * reduces dom(var) to {value}, then `tensorAC(Vars, [idx])` enforces arc
 * consistency with var as the only changed variable, so sweep 1 examines
 * only the constraints on var (Proposition 2) instead of every constraint.
 *
 *  dom_in      DEVICE, n_vars words: an ARC-CONSISTENT state (for example the
 *              result of an earlier enforcement).  Under that precondition the
 *              result, the removals of every sweep and the sweep count equal
 *              those of rac_enforce on the assigned state; without it the
 *              result may miss removals.
 *  var, value  the assignment, 0 <= var < n_vars, 0 <= value < d (a value
 *              outside dom_in[var] empties that domain: a wipe-out).
 *  dom_out, iterations, status, max_sweeps, flags, stream: as rac_enforce
 *              (dom_out receives the assigned and enforced state).
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
RAC_API rac_status rac_assign_enforce(const rac_network *net, const uint32_t *dom_in,
                                      uint32_t *dom_out, int32_t var, int32_t value,
                                      int32_t *iterations, int32_t *status, int32_t max_sweeps,
                                      uint32_t flags, rac_stream_t stream);

/*
 * rac_search -- the backtrack search of Algorithm 2 (`main` / `dfs`): enforce
 * arc consistency on the initial domains (`tensorAC(Vars, all)`), then pick
 * a variable, try its values in increasing order, and after each `assign`
 * enforce with only that variable changed (`tensorAC(Vars, [idx])`, as
 * rac_assign_enforce), descending while no domain is empty and backtracking
 * otherwise, until every domain is a singleton (a solution), every
 * assignment has been tried, or max_nodes assignments have been made.  The
 * variable order, which the paper leaves open (`heuristics()`), is the
 * smallest domain of size > 1, lowest index first.  The loop runs on the
 * host inside the library; every enforcement is one kernel launch that
 * writes its results straight into pinned host memory, and the call returns
 * when the search ends (it waits for `stream`).
 *
 *  dom0        HOST, n_vars words: the initial domains.
 *  max_nodes   assignments to make at most (>= 0).
 *  flags       RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL, for every enforcement.
 *  solution    HOST, n_vars words: receives the solution when one is found.
 *  found       HOST int32: 1 when a solution was found, else 0.
 *  exhausted   HOST int32: 1 when the search stopped at max_nodes.
 *  nodes       HOST int64: assignments made.
 *  root        HOST, 2 int32: sweep count and status of the root enforcement
 *              (the search stops at once unless the status is RAC_OK).
 *  steps       HOST, 5 x step_cap int32, or NULL with step_cap 0: per
 *              assignment in order, (level, variable, value, sweep count,
 *              status); level 0 is the first assignment below the root.
 * Device memory: one n_vars-word state per search level (allocated as the
 * search deepens, freed on return) and a pinned staging buffer.
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
RAC_API rac_status rac_search(const rac_network *net, const uint32_t *dom0, int64_t max_nodes,
                              uint32_t flags, rac_stream_t stream, uint32_t *solution,
                              int32_t *found, int32_t *exhausted, int64_t *nodes, int32_t *root,
                              int32_t *steps, int64_t step_cap);

/*
 * rac_enforce_batch -- many independent (network, domain state) items.
 *
 *  nets          HOST array of network handles.
 *  n_nets        entries in nets.
 *  n_items       number of items (>= 0).
 *  item_net      HOST, n_items int32: index into nets of each item.
 *  item_dom_off  HOST, n_items int64: word offset of the item's state in
 *                dom_in and dom_out (the state occupies that network's
 *                n_vars words).  Offsets may be in any order; the states of
 *                different items must not overlap.
 *  dom_in, dom_out  DEVICE word arrays (dom_out == dom_in allowed).
 *  iterations, status  DEVICE, n_items int32 each.
 *  max_sweeps, flags, stream  as for rac_enforce.
 *
 * Items on the same network are enforced together so that each relation
 * slab is read once per sweep for all of them.  When the items span several
 * networks, all of them run in ONE persistent launch (the batched kernel)
 * whose tables and scratch are allocated and freed in stream order around
 * the launch (cudaMallocAsync); for repeated batches over the same networks
 * a rac_plan avoids that per-call set-up.
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
RAC_API rac_status rac_enforce_batch(const rac_network *const *nets, int32_t n_nets, int32_t n_items,
                             const int32_t *item_net, const int64_t *item_dom_off,
                             const uint32_t *dom_in, uint32_t *dom_out, int32_t *iterations,
                             int32_t *status, int32_t max_sweeps, uint32_t flags,
                             rac_stream_t stream);

/*
 * rac_plan -- a fixed batch of (network, domain state) items enforced in one
 * persistent launch, with its tables and scratch allocated once.
 *
 * rac_plan_create: nets / n_nets / n_items / item_net / item_dom_off as for
 *   rac_enforce_batch (HOST arrays, copied).  Allocates device memory and
 *   synchronises with the device.  The networks must outlive the plan.
 * rac_plan_enforce: enforce every item (Eq. 1 to its fixpoint) in ONE
 *   cooperative launch on `stream`; dom_in / dom_out / iterations / status /
 *   max_sweeps / flags as for rac_enforce_batch.  Allocates nothing, so it can
 *   be captured in a CUDA graph.  Launches of one plan must not overlap on
 *   the GPU (use one plan per stream).
 * rac_plan_destroy: free the plan (NULL-safe; no launch of it may still run).
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
typedef struct rac_plan rac_plan;
RAC_API rac_status rac_plan_create(const rac_network *const *nets, int32_t n_nets,
                                   int32_t n_items, const int32_t *item_net,
                                   const int64_t *item_dom_off, rac_plan **out);
RAC_API rac_status rac_plan_enforce(rac_plan *plan, const uint32_t *dom_in, uint32_t *dom_out,
                                    int32_t *iterations, int32_t *status, int32_t max_sweeps,
                                    uint32_t flags, rac_stream_t stream);
RAC_API void rac_plan_destroy(rac_plan *plan);

/*
 * rac_enforce_host -- rac_enforce on HOST buffers: copies the n_states
 * states (n_states x n_vars words, state s at word s*n_vars) to the device,
 * enforces them as one batch on `net`, copies domains, iterations and status
 * back, and returns once they are in the caller's buffers.  The caller's
 * buffers (any host memory) are copied with memcpy to and from a pinned
 * staging buffer that the library allocates per (network, stream) and frees
 * in rac_destroy; the copy in, the launches and (calls of several launches,
 * or the tensor-core kernel) the copy out form a CUDA graph, recorded on the
 * first call with a given (n_states, max_sweeps, flags) and replayed by later
 * calls with the same ones.  A call of one bit-packed launch has the kernel
 * write its results straight into the pinned buffer; with at most three
 * states its last CTA then writes a completion number there, and the call
 * waits for that number instead of synchronising `stream` (the kernel's exit
 * may still be in flight when it returns; later work on `stream` is ordered
 * after it), synchronising `stream` only if the number does not come within
 * the wait limit.  Other calls synchronise `stream`.  Calls on the same (network, stream) must not
 * overlap.
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
RAC_API rac_status rac_enforce_host(const rac_network *net, int32_t n_states, const uint32_t *dom_in,
                            uint32_t *dom_out, int32_t *iterations, int32_t *status,
                            int32_t max_sweeps, uint32_t flags, rac_stream_t stream);

/*
 * rac_enforce_noalloc -- rac_enforce without any device allocation.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc while they enforce, such as processes whose device memory
 * is entirely reserved by another allocator (a framework's caching pool), or
 * latency-bound loops that cannot take the device-wide synchronisation that
 * cudaMalloc/cudaFree may imply.
 *
 * Arguments, results and errors are those of rac_enforce with the bit-packed
 * kernel; RAC_KERNEL_TENSOR is refused with RAC_ENOTSUP.  The scratch space
 * is one static array inside the library (311,808 bytes, about 305 KiB, on
 * every device that loads it, held until the process exits), so:
 *  - networks with more than RAC_NOALLOC_MAX_VARS variables are rejected with
 *    RAC_EINVAL and an explanatory rac_last_error();
 *  - all calls share the array: calls whose kernels overlap on the GPU (other
 *    streams, other host threads) race and give undefined results;
 *  - every call resets the array on its stream first, sticky error word
 *    included: a call whose bounded wait ran out (status RAC_EBARRIER) does
 *    not poison later calls, unlike rac_enforce's per-stream workspace;
 *  - the first call on a device, with that device current, looks up the
 *    array's device address, and the first call for each relation width
 *    (d rounded up to a multiple of 4) on a device sets that kernel's
 *    launch attributes; make those first calls before starting any stream
 *    capture.
 */
#define RAC_NOALLOC_MAX_VARS 65536
RAC_API rac_status rac_enforce_noalloc(const rac_network *net, const uint32_t *dom_in,
                                       uint32_t *dom_out, int32_t *iterations, int32_t *status,
                                       int32_t max_sweeps, uint32_t flags, rac_stream_t stream);

/* ---------------------------------------------------------------------------
 * Partitioned sweep of one network over several ranks (one process per GPU).
 *
 * Eq. 1 (Sec. 3) computes every D^(k)[x] from D^(k-1) alone, and a sweep keeps
 * (x,a) only if it has a support on EVERY constraint of C_x: an AND over the
 * constraints.  So when the constraints are split over G ranks, rank g's one
 * sweep of its share (rac_enforce on a network made of those constraints,
 * max_sweeps = 1, input D^(k-1)) gives a partial next domain
 * P_g = D^(k-1) AND (supports on its share), and D^(k) = AND_g P_g exactly.
 * The ranks all-gather their partials (G x n_vars words) and each combines
 * them with this call; the loop's decisions (some domain changed, some
 * domain empty) come from the gathered words, identical on every rank, so
 * no second collective is needed.
 *
 * rac_combine_partials -- dom_next[x] = dom_prev[x] AND partials[g][x] for
 * g < n_parts; flags[0] = 1 iff some dom_next[x] != dom_prev[x], flags[1] =
 * 1 iff some dom_next[x] == 0 (an empty domain), else 0.
 *
 *  partials    DEVICE, n_parts x n_vars words, part g at word g * n_vars (the
 *              layout of an all-gather of the ranks' partials).
 *  dom_prev    DEVICE, n_vars words: D^(k-1).
 *  dom_next    DEVICE, n_vars words: receives D^(k).  dom_next == dom_prev is
 *              allowed; no other overlap with either input is.
 *  flags       DEVICE, 2 int32 (cleared and written on `stream`).
 * Errors: RAC_EINVAL (n_parts < 1, n_vars < 0, a NULL pointer), RAC_ECUDA.
 */
RAC_API rac_status rac_combine_partials(int32_t n_parts, int32_t n_vars, const uint32_t *partials,
                                        const uint32_t *dom_prev, uint32_t *dom_next,
                                        int32_t *flags, rac_stream_t stream);

/* ---------------------------------------------------------------------------
 * Learned active-block gating.
 *
 * The paper gates sweeps exactly with Proposition 2 (Sec. 3): sweep k >= 2
 * only needs the constraints touching a variable whose domain changed in
 * sweep k-1.  On dense networks that set is nearly every relation slab, yet
 * most of those evaluations remove nothing.  A small learned predictor
 * scores each (slab, state) candidate before it is evaluated and skips the
 * unpromising ones; a skipped pair stays PENDING until a sweep evaluates it.
 * Exactness is kept by the recurrence itself:
 *  - every removal is made from a superset of D_ac, hence sound (Lemma 1);
 *  - a gated sweep that removes nothing is followed by a verification sweep
 *    that evaluates, without the predictor, every pending pair and every
 *    Proposition-2 candidate.  A pair that is neither has been evaluated
 *    since the last change of any of its variables and removed nothing
 *    then, so it would remove nothing now (Proposition 2's argument): a
 *    sweep that removes nothing and leaves no pair pending is equivalent to
 *    a full sweep that removes nothing.  Only such a sweep ends a state; its
 *    domain is arc consistent and contains D_ac, i.e. it is D_ac.
 *  - with RAC_VERIFY_FULL the verification sweep evaluates every slab
 *    literally, and only a full sweep that removes nothing ends a state.
 * So the result and status are those of rac_enforce; the sweep count is the
 * number of sweeps this gated recurrence executed (it may differ).
 *
 * Every sweep is gated, the first one included: before sweep 1 a variable
 * counts as changed when its input domain is not full (so on states that
 * assign a few variables of full domains the predictor can learn the seeded
 * first sweep of Algorithm 2; nothing relies on it).
 *
 * The predictor is an MLP 8 -> 64 -> 64 -> 1 (ReLU hidden layers, a logit
 * out) with BF16 weights and FP32 accumulation.  Its 8 features of a (slab,
 * state) pair before sweep k, all in [0, 1]:
 *   f0 min(k, 16) / 16; f1 slab rows (variables x) changed in sweep k-1 /
 *   slab rows; f2 column-block variables y changed in sweep k-1 / 32; f3 the
 *   slab's disallowed fraction of relation bits (tightness); f4 constraints
 *   in the slab / (slab rows * 32); f5 min over the column variables of
 *   |D_{k-1}(y)| / d; f6 mean of the same; f7 min over the slab's row
 *   variables of |D_{k-1}(x)| / d.
 * Parameters (RAC_PREDICTOR_PARAMS floats, in this order): W1[64][8], b1[64],
 * W2[64][64], b2[64], w3[64], b3.  Forward: x~ = bf16(x), h1 = bf16(relu(W1
 * x~ + b1)), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3.
 * ------------------------------------------------------------------------- */
typedef struct rac_predictor rac_predictor;
#define RAC_PREDICTOR_FEATURES 8
#define RAC_PREDICTOR_PARAMS 4801

/* rac_predictor_num_params -- RAC_PREDICTOR_PARAMS. */
RAC_API int32_t rac_predictor_num_params(void);

/* rac_predictor_create -- a predictor on the current device, He-initialised
 * from `seed` (biases zero).  Synchronises with the device.
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA. */
RAC_API rac_status rac_predictor_create(uint64_t seed, rac_predictor **out);

/* rac_predictor_destroy -- NULL-safe; no launch using it may still run. */
RAC_API void rac_predictor_destroy(rac_predictor *p);

/* rac_predictor_set_weights / rac_predictor_get_weights -- HOST arrays of
 * RAC_PREDICTOR_PARAMS floats.  set: replaces the FP32 master weights (and
 * their BF16 copy), resets the optimiser state.  get: the FP32 master
 * weights, or with bf16 != 0 the BF16 copy that inference uses, widened.
 * Both synchronise with the device.  Errors: RAC_EINVAL, RAC_ECUDA. */
RAC_API rac_status rac_predictor_set_weights(rac_predictor *p, const float *params);
RAC_API rac_status rac_predictor_get_weights(const rac_predictor *p, float *params, int32_t bf16);

/* rac_predictor_gradient -- mean loss and its gradient over n samples.
 *  x      DEVICE, n x 8 floats (features); y DEVICE, n floats (labels 0/1).
 *  Loss per sample: w(y) (softplus(z) - y z), w(1) = pos_weight, w(0) = 1.
 *  The gradient is taken at the BF16 weights, with the BF16 rounding of x and
 *  h1 passed straight through.
 *  grad   HOST, RAC_PREDICTOR_PARAMS floats (may be NULL); loss HOST (may be
 *  NULL).  Synchronises.  Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA. */
RAC_API rac_status rac_predictor_gradient(rac_predictor *p, const float *x, const float *y,
                                          int64_t n, float pos_weight, float *grad, float *loss);

/* rac_predictor_train -- `steps` Adam steps (beta1 0.9, beta2 0.999, eps
 * 1e-8, learning rate lr) on minibatches of `batch` samples drawn uniformly
 * with replacement from the n samples (x, y as above, DEVICE), the draws
 * fixed by `seed`.  loss (HOST, may be NULL) receives the last minibatch's
 * loss.  Synchronises.  Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA. */
RAC_API rac_status rac_predictor_train(rac_predictor *p, const float *x, const float *y, int64_t n,
                                       int32_t steps, int32_t batch, float lr, float pos_weight,
                                       uint64_t seed, float *loss);

/* rac_predictor_predict -- logits of n samples (x DEVICE n x 8, logits
 * DEVICE n).  tensor_cores != 0 runs the warp-wide tensor-core routine the
 * sweep kernel uses, 0 a scalar one.  Synchronises.
 * Errors: RAC_EINVAL, RAC_ECUDA. */
RAC_API rac_status rac_predictor_predict(const rac_predictor *p, const float *x, int64_t n,
                                         float *logits, int32_t tensor_cores);

/* Optional record of the gating decisions of rac_enforce_learned: one record
 * per Proposition-2 candidate (slab, state) of every sweep (sweep 1: every
 * pair; with a predictor, candidates of verification sweeps too; pending
 * pairs that are no candidate get no record).  Records are appended in no
 * particular order. */
typedef struct rac_trace {
  float *features;   /* DEVICE, capacity x 8: the features above */
  float *label;      /* DEVICE, capacity: 1 the evaluation removed a value,
                        0 it did not, -1 the pair was skipped */
  float *logit;      /* DEVICE, capacity (may be NULL): the predictor's logit,
                        NaN without a predictor */
  int32_t *where;    /* DEVICE, capacity x 4: sweep k (| 1 << 30 if the state
                        was in its gated phase), state index, tile I | J << 16
                        (rows of variables 32 I.., columns 32 J..), rows
                        row0 | nrows << 8 (slab rows inside the tile) */
  int64_t capacity;  /* records that fit (0: count only) */
  unsigned long long *count;      /* DEVICE (may be NULL): records offered, may
                                     exceed capacity; set to 0 by the call */
  unsigned long long *evaluated;  /* DEVICE (may be NULL): (slab, state)
                                     evaluations executed in all sweeps; set to
                                     0 by the call */
} rac_trace;

/*
 * rac_enforce_learned -- rac_enforce for n_states states (state s at word
 * s * n_vars of dom_in / dom_out, DEVICE), with learned gating.
 *
 *  pred       the predictor, or NULL: then every sweep k >= 2 evaluates
 *             exactly the Proposition-2 candidates (as RAC_INCREMENTAL), the
 *             mode used to record training traces.
 *  threshold  a candidate of a gated sweep is evaluated iff its logit >
 *             threshold.
 *  min_scored the states are scored 32 at a time per slab; a 32-state group
 *             with fewer than min_scored gated candidates on a slab is not
 *             scored and all its candidates are evaluated (the predictor's
 *             cost per slab would exceed what it can save).  <= 1: always
 *             score.
 *  sweeps     DEVICE, n_states int32: sweeps executed.
 *  status     DEVICE, n_states int32: as rac_enforce (identical values).
 *  max_sweeps, stream: as rac_enforce.  flags: RAC_STOP_ON_WIPEOUT (the
 *             returned domain is then the state at the first sweep that
 *             emptied a domain -- a sound superset of D_ac, not unique),
 *             RAC_VERIFY_FULL (see above).
 *  trace      optional (NULL: none).
 * Errors: RAC_EINVAL, RAC_ENOMEM, RAC_ECUDA.
 */
RAC_API rac_status rac_enforce_learned(const rac_network *net, int32_t n_states,
                                       const uint32_t *dom_in, uint32_t *dom_out, int32_t *sweeps,
                                       int32_t *status, int32_t max_sweeps, uint32_t flags,
                                       const rac_predictor *pred, float threshold,
                                       int32_t min_scored, const rac_trace *trace,
                                       rac_stream_t stream);

/*
 * rac_network_info -- describe a network: writes up to n_info int64 values
 * to info, in this order: n_vars, d, n_cons, relation-slab bytes on the
 * device, number of relation slabs, rows per slab, words per stored relation
 * (round_up(d, 4), or ceil(round_up(d, 4)^2 / 32) with RAC_LAYOUT_PACKED and
 * d <= 28).  Returns the number written.
 */
RAC_API int32_t rac_network_info(const rac_network *net, int64_t *info, int32_t n_info);

/* rac_last_error -- message for the last failing call on this host thread
 * ("" if none).  The string stays valid until the next call on the thread. */
RAC_API const char *rac_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RAC_H */
