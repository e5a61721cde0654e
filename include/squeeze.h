/*
 * squeeze.h -- C ABI of the GB300 compact-fractal library.
 *
 * The library runs the neighbourhood step of Squeeze (Quezada, Navarro,
 * Hitschfeld, Bustos, arXiv 2201.00613) on an NBB fractal that is stored only
 * in compact form: lambda maps a compact index to expanded space (Sec. 3.3),
 * the neighbours (the 8 Moore neighbours unless another neighbourhood is set)
 * are formed there, nu maps each back to a compact index or rejects it as a
 * hole (Sec. 3.4), and a Life-like rule writes the next state into a second
 * compact buffer (Sec. 4).  Comparators (bounding box, the lambda(omega)
 * approach, the block-level layout, tensor-core maps) and other workloads
 * (heat diffusion, Ising spins) share the same handle.  Three-dimensional
 * fractals have a handle of their own (squeeze_3d_*); checkpoint files of a
 * compact state are written and read by host-only calls.
 *
 * Conventions for every entry point:
 *   - Return value: SQUEEZE_OK (0) or a negative SQUEEZE_ERR_* code.  Nothing
 *     throws, exits or traps; squeeze_status_string() describes a code.
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *     pointers owned by the caller.  The library keeps no reference to either
 *     after the call returns, except a batch, which keeps its items' buffers
 *     until squeeze_batch_destroy().
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  Argument errors are reported synchronously;
 *     errors found on the device are latched in a per-handle status word and
 *     reported by squeeze_device_status().
 *   - The handle owns small per-fractal tables and, once the tiled step has
 *     run, its neighbour program and adjacency table (4 bytes per tile and
 *     direction) in device memory, freed by squeeze_destroy().  squeeze_step
 *     also keeps two border-record buffers of 4 bytes per 32 halo cells of a
 *     tile (1/30 of a state for the triangle, 1/4 for the carpet with eight
 *     steps per launch); a batch keeps its own per item.
 *   - Calls that use one handle must be ordered on the GPU (one stream, or
 *     streams ordered by events): its status word and record buffers are
 *     shared by its calls.
 *
 * Compact layout (Sec. 3.1): level mu odd unrolls along x, even along y, so
 * the compact rectangle has W = k^ceil(r/2) columns and H = k^floor(r/2)
 * rows, stored row-major: omega = w_y * W + w_x.  A state buffer holds k^r
 * bytes, one per fractal cell; a cell is alive iff bit 0 of its byte is set
 * (the other bits are ignored), and the library writes only 0 and 1.
 */
#ifndef SQUEEZE_H
#define SQUEEZE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SQUEEZE_OK 0
#define SQUEEZE_ERR_INVALID_ARG (-1)   /* bad pointer, size, descriptor or kind   */
#define SQUEEZE_ERR_UNSUPPORTED (-2)   /* valid request this build cannot serve   */
#define SQUEEZE_ERR_OOM (-3)           /* device or host allocation failed        */
#define SQUEEZE_ERR_CUDA (-4)          /* a CUDA runtime call failed              */
#define SQUEEZE_ERR_DEVICE_TIMEOUT (-5) /* a bounded device-side wait gave up     */
#define SQUEEZE_ERR_DEVICE_BOUNDS (-6) /* a device-side bounds check fired        */
#define SQUEEZE_ERR_IO (-7)            /* a file could not be read or written, or is damaged */
#define SQUEEZE_ERR_DEVICE_UNSAFE (-8) /* a timed-out bulk copy never landed: later launches on
                                          this context may see it land in their shared memory */

/* ---- fault injection (tests of the error paths) --------------------------- */
#define SQUEEZE_FAULT_WITHHOLD_LOADS 1u  /* tiled kernel issues no bulk loads: its waits run out */

/* ---- step kernels --------------------------------------------------------- */
#define SQUEEZE_STEP_AUTO 0    /* tiled kernel when the level allows, else per-cell ALU */
#define SQUEEZE_STEP_TILED 1   /* bit-sliced tile kernel (self-similar neighbour program) */
#define SQUEEZE_MAP_ALU 2      /* one thread per cell: integer lambda + 8 nu (Sec. 3.2)  */
#define SQUEEZE_MAP_TC_BF16 3  /* one thread per cell, map sums on tcgen05 kind::f16    */
#define SQUEEZE_MAP_TC_I8 4    /* tcgen05 kind::i8: not available on sm_103a            */

typedef struct squeeze_handle squeeze_handle;

/* squeeze_create -- describe a level-r NBB fractal F_n^{k,s} (Sec. 3).
 *   s        growth factor per level, 2 <= s <= 16.
 *   k        replicas per level, 1 <= k <= min(s*s, 255).
 *   offsets  host array of 2*k bytes: replica beta sits at (tau_x, tau_y) =
 *            (offsets[2*beta], offsets[2*beta+1]), each < s, all pairs
 *            distinct (Eq. tau; the replica order fixes the compact order).
 *   r        level; requires s^r <= 2^30 and W, H < 2^32.
 *   out      receives the new handle.
 * Errors: INVALID_ARG for any violated bound; OOM / CUDA when the device
 * tables cannot be allocated on the current device. */
int squeeze_create(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                   squeeze_handle **out);

/* squeeze_destroy -- free the handle's device tables.  Synchronises the
 * device first.  NULL is accepted. */
int squeeze_destroy(squeeze_handle *h);

/* squeeze_info -- sizes of the fractal (Sec. 3, Eq. V and Sec. 3.1).
 *   n_cells = k^r; width = W; height = H; side = n = s^r.  Any output pointer
 *   may be NULL. */
int squeeze_info(const squeeze_handle *h, uint64_t *n_cells, uint64_t *width,
                 uint64_t *height, uint64_t *side);

/* squeeze_set_rule -- birth/survive masks of the outer-totalistic rule:
 * a dead cell with c alive fractal neighbours becomes alive iff bit c of
 * `birth` is set; an alive cell stays alive iff bit c of `survive` is set.
 * Default B3/S23: birth = 1<<3, survive = (1<<2)|(1<<3) (Sec. 4).  Masks must
 * fit in 9 bits.  Affects steps enqueued after the call. */
int squeeze_set_rule(squeeze_handle *h, uint32_t birth, uint32_t survive);

/* squeeze_lambda -- compact -> expanded map (Sec. 3.3, Eqs. lambda, beta).
 *   d_omega  count linear compact indices (uint64).
 *   d_xy     receives 2*count int32: (x, y) per index; (-1, -1) for an index
 *            >= k^r.
 * Both arrays must be 8-byte aligned (else INVALID_ARG).  Uses the integer
 * ALU form. */
int squeeze_lambda(const squeeze_handle *h, const uint64_t *d_omega, int32_t *d_xy,
                   uint64_t count, void *stream);

/* squeeze_nu -- expanded -> compact map with hole rejection (Sec. 3.4,
 * Eqs. theta, t, f, nux, nuy; theta read as the base-s digit mu-1 and odd
 * levels accumulated on x, which makes nu the inverse of lambda).
 *   d_xy     2*count int32 points (x, y); any value is allowed.
 *   d_omega  receives count uint64: the compact index, or UINT64_MAX for a
 *            hole or a point outside [0, s^r)^2.
 * Both arrays must be 8-byte aligned (else INVALID_ARG). */
int squeeze_nu(const squeeze_handle *h, const int32_t *d_xy, uint64_t *d_omega,
               uint64_t count, void *stream);

/* squeeze_map_tc -- the same two maps with their digit-times-weight sums run
 * as tcgen05 matrix multiplies (Sec. 3.6).  kind = SQUEEZE_MAP_TC_BF16: the
 * per-level digits (tau components for lambda, replica ids for nu; all < 256)
 * are bf16 rows of A, the level weights (s^(mu-1) for lambda; k^((mu-1)/2) or
 * W k^((mu-2)/2) for nu) are split into radix-256 limbs as the columns of B,
 * and fp32 accumulates each column.  Exact: with r <= 30 and every digit and
 * limb <= 255 a column sum is below 30 * 254 * 255 < 2^21 < 2^24, so fp32
 * holds every partial sum exactly in any order; limbs are recombined in
 * 64-bit integers.  kind = SQUEEZE_MAP_TC_I8 returns UNSUPPORTED (the integer
 * MMA kind is not available on sm_103a).
 *   direction 0: lambda (d_in = count uint64 omega, d_out = count int32 xy
 *                pairs, (-1, -1) for omega >= k^r);
 *   direction 1: nu (d_in = count int32 xy pairs, d_out = count uint64
 *                omega, UINT64_MAX for a hole or a point off the box).
 * Same outputs as squeeze_lambda / squeeze_nu.  Both pointers 8-byte aligned
 * (else INVALID_ARG); count = 0 enqueues nothing. */
int squeeze_map_tc(const squeeze_handle *h, int direction, const void *d_in, void *d_out,
                   uint64_t count, int kind, void *stream);

/* squeeze_init_bernoulli -- seeded Bernoulli initial state in compact order.
 * Cell omega with expanded position (x, y) = lambda(omega) is alive iff
 * (SplitMix64 output number (y*2^32 + x) of the stream seeded with `seed`)
 * >> 40 is below p_q24 (= floor(p * 2^24)); SplitMix64 as published by
 * Steele, Lea and Flood (OOPSLA 2014).  Keying by expanded position makes the
 * state independent of the replica order.
 *   d_state  k^r bytes, written with 0/1. */
int squeeze_init_bernoulli(const squeeze_handle *h, uint8_t *d_state, uint64_t seed,
                           uint32_t p_q24, void *stream);

/* squeeze_step -- n_steps synchronous rule steps on the compact state
 * (Sec. 3.2 neighbourhood exploration, Sec. 4 automaton): holes and points
 * outside the box are dead neighbours; no wrap.
 *   d_buf0   k^r bytes, the current state (read on even steps).
 *   d_buf1   k^r bytes, scratch for the other parity.
 *   The result is in d_buf0 when n_steps is even and in d_buf1 when odd.
 *   kind     SQUEEZE_STEP_* / SQUEEZE_MAP_*.  TC_I8 -> UNSUPPORTED.
 * The two buffers must not overlap.  n_steps = 0 enqueues nothing.  The tiled
 * kernel needs both buffers 16-byte aligned (its bulk copies): TILED with a
 * misaligned buffer is INVALID_ARG, and AUTO then takes the per-cell ALU
 * kernel.  A level whose tiled program would not fit is UNSUPPORTED for
 * TILED (AUTO falls back to the per-cell ALU kernel only when no tile level
 * fits at all).  squeeze_last_step_info() tells which kernel AUTO chose.
 * The tiled kernel advances up to eight steps per launch where its program
 * allows (the intermediate states stay in shared memory), so d_buf1 holds no
 * particular step afterwards; the result is the same bit for bit. */
int squeeze_step(squeeze_handle *h, uint8_t *d_buf0, uint8_t *d_buf1, uint64_t n_steps,
                 int kind, void *stream);

/* squeeze_record_bytes -- bytes of one border-record buffer of the handle's
 * tiled program (0 when its tiles have no halo): the states of the cells that
 * adjacent tiles read as halo, 4 bytes per 32 such cells and direction per
 * tile.  Prepares the tiled program if needed. */
int squeeze_record_bytes(squeeze_handle *h, uint64_t *bytes);

/* squeeze_write_records -- the border records of the compact state d_state
 * (16-byte aligned) into d_rec (squeeze_record_bytes bytes, 4-byte aligned),
 * one launch on `stream`; nothing for a program without records. */
int squeeze_write_records(squeeze_handle *h, const uint8_t *d_state, uint32_t *d_rec,
                          void *stream);

/* squeeze_set_max_steps_per_launch -- the most steps one launch of the tiled
 * kernel may advance: 1, 2, 4 or 8, or 0 for the default (the most whose
 * kernel keeps the CTAs per SM of the one-step kernel, or 3 if that has
 * more; its shared memory grows with the halo rings each further step
 * needs).  The result of squeeze_step
 * does not depend on it.  INVALID_ARG for other values. */
int squeeze_set_max_steps_per_launch(squeeze_handle *h, uint32_t steps);

/* squeeze_last_step_info -- what the handle's last accepted squeeze_step
 * call ran: *kind = SQUEEZE_STEP_TILED, SQUEEZE_MAP_ALU or SQUEEZE_MAP_TC_BF16
 * (0 before the first step), so that a caller of AUTO can see a fall-back to
 * the per-cell ALU kernel (misaligned buffers; about 300x slower than the
 * tiled kernel); *launches = kernel launches it enqueued; by_steps[i] (four
 * entries) = how many of them advanced 2^i steps (the tiled kernel runs n
 * steps as launches of 8, 4, 2 and 1 steps whose count has the parity of n:
 * n = 100 is 12 launches of 8 steps and 2 of 2).  *launches also counts one
 * launch that writes the border records of the input (the halo the first
 * step reads), which advances no step (none for a fractal whose tiles have no
 * halo).  Any pointer may be NULL.
 * INVALID_ARG for a null handle. */
int squeeze_last_step_info(const squeeze_handle *h, int *kind, uint64_t *launches,
                           uint64_t *by_steps);

/* squeeze_step_host -- the same run from and to HOST memory: copies h_in
 * (k^r bytes, ideally pinned) into d_buf0, runs n_steps, copies the result to
 * h_out (k^r bytes), all on `stream`, then synchronises the stream.
 * d_buf0 / d_buf1 are caller-owned device work buffers of k^r bytes. */
int squeeze_step_host(squeeze_handle *h, const uint8_t *h_in, uint8_t *h_out,
                      uint8_t *d_buf0, uint8_t *d_buf1, uint64_t n_steps, int kind,
                      void *stream);

/* squeeze_tiled_level -- the tile level L the tiled kernel uses for this
 * handle (a tile is one level-L sub-replica, k^L cells, stored as a
 * k^ceil(L/2) x k^floor(L/2) compact rectangle), or a negative code when the
 * tiled kernel is not available (then AUTO runs the per-cell ALU kernel).
 * squeeze_set_tiled_level() overrides the choice: 0 < L <= r, else
 * INVALID_ARG; a tile row wider than 32 cells (k^ceil(L/2) > 32) other than
 * exactly 64 cells, or a level whose tile program does not fit the kernel's
 * shared memory, gives UNSUPPORTED. */
int squeeze_tiled_level(const squeeze_handle *h);
int squeeze_set_tiled_level(squeeze_handle *h, uint32_t level);

/* ---- expanded bounding-box comparator (Sec. 4, approach "BB") ------------
 * The same automaton on the n x n expanded grid, one byte per cell:
 * bit 0 = alive, bit 1 = fractal cell; holes are 0 and stay 0.  Grids hold
 * n*n bytes, row-major (y * n + x). */

/* squeeze_bb_init -- Bernoulli start on the box, identical cell by cell to
 * squeeze_init_bernoulli (same seed / p_q24 give the same alive cells). */
int squeeze_bb_init(const squeeze_handle *h, uint8_t *d_grid, uint64_t seed, uint32_t p_q24,
                    void *stream);

/* squeeze_bb_step -- n_steps steps on the box; result in d_grid0 when n_steps
 * is even, d_grid1 when odd. */
int squeeze_bb_step(const squeeze_handle *h, uint8_t *d_grid0, uint8_t *d_grid1,
                    uint64_t n_steps, void *stream);

/* ---- other neighbourhoods and a PDE (Sec. 1) -------------------------------
 * Sec. 1 names stencil simulations, cellular automata and PDE solvers as the
 * uses of the compact maps. */

/* squeeze_set_neighbourhood -- the neighbourhood every step counts over: a
 * 9-bit mask over the 3 x 3 block, bit (dy+1)*3 + (dx+1) selecting offset
 * (dx, dy); SQUEEZE_MOORE (the default) or SQUEEZE_VON_NEUMANN, or any other
 * set of offsets.  Bit 4 (the cell itself) must be 0; masks of 9 or more
 * bits are INVALID_ARG.  Rebuilds the tiled program on the next tiled step. */
#define SQUEEZE_MOORE 0x1EF
#define SQUEEZE_VON_NEUMANN 0xAA
int squeeze_set_neighbourhood(squeeze_handle *h, uint32_t mask);

/* squeeze_heat_step -- n_steps explicit Euler steps of the heat equation on
 * the fractal graph, in fp32: u'(p) = u(p) + alpha * sum over the fractal
 * neighbours q of p (the handle's neighbourhood) of (u(q) - u(p)).  Holes and
 * points off the box have no edge, so the sum of u is conserved; with
 * alpha * (neighbours) <= 1 no value leaves the range of the start.
 *   d_u0, d_u1  k^r floats each, 4-byte aligned, not overlapping; the result
 *               is in d_u0 when n_steps is even and in d_u1 when odd. */
int squeeze_heat_step(const squeeze_handle *h, float *d_u0, float *d_u1, uint64_t n_steps,
                      float alpha, void *stream);

/* squeeze_ising_sweep -- n_sweeps checkerboard Metropolis sweeps of Ising
 * spins (coupling 1) on the fractal graph, in place: spin +1 where bit 0 of
 * d_state (k^r bytes) is set, and the result is written as 0/1.  A sweep
 * updates the cells with x + y even, then those with x + y odd; half-sweep
 * number t of the call (t = 0 .. 2 n_sweeps - 1) draws from the SplitMix64
 * stream seeded with SplitMix64 output t of `seed`, cell (x, y) taking output
 * y * 2^32 + x.  With dE = 2 s * (sum of neighbour spins) the spin flips iff
 * dE <= 0 or (draw >> 40) < floor(exp(-dE / temperature) * 2^24).  The
 * handle's neighbourhood must join only cells of opposite parity (a subset
 * of von Neumann; else UNSUPPORTED); temperature >= 0 (0: only dE <= 0
 * flips; else INVALID_ARG).  Give each call its own seed. */
int squeeze_ising_sweep(const squeeze_handle *h, uint8_t *d_state, uint64_t n_sweeps,
                        uint64_t seed, double temperature, void *stream);

/* squeeze_lambda_step -- the lambda(omega) approach on the same box (Sec. 2):
 * one thread per compact index omega maps it with lambda and reads its 8
 * neighbours directly in the box, so no nu is needed but the memory is the
 * whole n x n box.  Same box format as squeeze_bb_step (bit 0 alive, bit 1
 * fractal cell, holes 0) and the same results.  Only fractal cells are
 * written: the holes of d_grid1 must already be 0 (for instance a copy of
 * the initial d_grid0).  The result is in d_grid0 when n_steps is even and
 * in d_grid1 when odd; the grids must differ (else INVALID_ARG). */
int squeeze_lambda_step(const squeeze_handle *h, uint8_t *d_grid0, uint8_t *d_grid1,
                        uint64_t n_steps, void *stream);

/* squeeze_bb_to_compact -- gather the alive bits of the box into compact order
 * (d_state, k^r bytes of 0/1), for comparing the two representations. */
int squeeze_bb_to_compact(const squeeze_handle *h, const uint8_t *d_grid, uint8_t *d_state,
                          void *stream);

/* ---- batched steps over many fractals -------------------------------------
 * A batch steps many independent instances (any mix of NBB fractals and
 * levels, each with its own handle, rule and buffer pair) together.  The
 * items are split by the tiled kernel's tile-row instantiation (tile rows of
 * 27, 25, 64, ... cells); one CA step of all of them is one launch of a
 * persistent kernel per instantiation, whose CTAs walk a balanced schedule
 * of (instance, group range) entries (balanced by group slots, since a
 * group costs about the same whether its 32 tiles are all present).  The
 * paper has no batched form; its step (Sec. 3.2, Sec. 4) is applied to each
 * instance unchanged, so every result equals the instance's own
 * squeeze_step with SQUEEZE_STEP_TILED. */
typedef struct squeeze_batch squeeze_batch;
typedef struct {
  squeeze_handle *h;  /* the instance's fractal, level and rule */
  uint8_t *d_buf0;    /* k^r bytes, 16-byte aligned: the state (even steps) */
  uint8_t *d_buf1;    /* k^r bytes, 16-byte aligned, not overlapping d_buf0 */
} squeeze_batch_item;

/* squeeze_batch_create -- validate the items, prepare every handle's tiled
 * program, build the schedule and copy the descriptors to the device.  The
 * handles' rules and tile levels are read now: later changes need a new
 * batch.  The handles and buffers must outlive the batch.  INVALID_ARG for a
 * null, misaligned or overlapping item; UNSUPPORTED when the items' programs
 * together need more shared memory than one CTA may use; OOM / CUDA when a
 * device allocation or copy fails (nothing is left allocated then). */
int squeeze_batch_create(const squeeze_batch_item *items, uint32_t count, squeeze_batch **out);

/* squeeze_batch_create_with_records -- squeeze_batch_create with the items'
 * border records in the caller's buffers: d_rec[2 i] holds the records of
 * item i's d_buf0 and d_rec[2 i + 1] those of its d_buf1, squeeze_record_bytes
 * bytes each (4-byte aligned; ignored, and may be null, for an item whose
 * program has none).  The records of every d_buf0 must be current (written by
 * squeeze_write_records, or by a run of a batch that used the same buffers),
 * so the first run makes no records-only launch; runs keep each item's records
 * in step with its states.  Errors as squeeze_batch_create, and INVALID_ARG for
 * a missing or misaligned record buffer. */
int squeeze_batch_create_with_records(const squeeze_batch_item *items, uint32_t count,
                                      uint32_t *const *d_rec, squeeze_batch **out);

/* squeeze_batch_configure -- launch shape chosen by the autotuner: threads per
 * CTA (0 = each instantiation's own choice, the one squeeze_step makes; else a
 * multiple of 32 in 64..384 for every launch), CTAs per SM (0 = as many as
 * fit) and whether squeeze_batch_run replays a captured CUDA graph (1) or
 * launches directly.  The default is (0, 0, 1). */
int squeeze_batch_configure(squeeze_batch *b, uint32_t threads, uint32_t ctas_per_sm,
                            int use_graph);

/* squeeze_batch_info -- the resulting launch shape: the CTAs of one step
 * (summed over the instantiations' launches), the largest CTA size and the
 * largest dynamic shared memory of a launch. */
int squeeze_batch_info(const squeeze_batch *b, uint32_t *grid, uint32_t *threads,
                       uint32_t *smem_bytes);

/* squeeze_batch_run -- n_steps steps of every instance on `stream`, one
 * launch per instantiation and group of 1, 2, 4 or 8 steps (up to eight
 * steps per launch where the programs allow; the launch count keeps the
 * parity of n_steps), after one launch per instantiation that writes the
 * border records of the states (the halo of the first step) unless the
 * previous run of the batch left them current; with graphs on, the launches
 * are captured once (per distinct n_steps, starting buffer and whether the
 * records are written) and replayed.  The batch keeps the step count across
 * calls: every instance's state is in d_buf0 after an even total number of
 * steps since squeeze_batch_create and in d_buf1 after an odd one.  Between
 * runs the batch owns its items' states: a caller that writes one calls
 * squeeze_batch_states_written before the next run. */
int squeeze_batch_run(squeeze_batch *b, uint64_t n_steps, void *stream);

/* squeeze_batch_states_written -- the caller wrote items' states after the
 * last run: the next run rewrites the border records first.  INVALID_ARG for
 * a null batch. */
int squeeze_batch_states_written(squeeze_batch *b);

/* squeeze_batch_destroy -- free the batch (not the handles or buffers). */
int squeeze_batch_destroy(squeeze_batch *b);

/* ---- block-level layout (Sec. 3.5) ----------------------------------------
 * With rho = s^b, the state is stored as k^(r-b) blocks in the compact order
 * of level r - b (row-major, k^ceil((r-b)/2) blocks per row), each block the
 * rho x rho expanded micro-box of its level-b sub-replica, holes included as
 * 0: k^(r-b) * rho^2 bytes (one byte per cell, alive iff bit 0).  b = 0 is
 * the compact layout.  b must satisfy b <= r (else INVALID_ARG), rho <= 32
 * and k^(r-b) < 2^32 blocks (else UNSUPPORTED).  The paper has this layout as its block
 * variant of Squeeze; the results equal those of the compact layout. */

/* squeeze_block_bytes -- bytes of one block-layout state at level b. */
int squeeze_block_bytes(const squeeze_handle *h, uint32_t b, uint64_t *bytes);

/* squeeze_block_init -- the seeded Bernoulli start of squeeze_init_bernoulli
 * (same cells alive) in block layout; micro-box holes are written as 0. */
int squeeze_block_init(const squeeze_handle *h, uint32_t b, uint8_t *d_blocks, uint64_t seed,
                       uint32_t p_q24, void *stream);

/* squeeze_block_step -- n_steps rule steps in block layout (one thread per
 * micro-box cell; neighbours across a block border through the 8 adjacent
 * blocks, found by the carry walk of nu at block level).  Result in d_blocks0
 * when n_steps is even, d_blocks1 when odd; the buffers must differ. */
int squeeze_block_step(const squeeze_handle *h, uint32_t b, uint8_t *d_blocks0,
                       uint8_t *d_blocks1, uint64_t n_steps, void *stream);

/* squeeze_block_to_compact -- the same state in compact order (k^r bytes of
 * 0/1), for comparing layouts. */
int squeeze_block_to_compact(const squeeze_handle *h, uint32_t b, const uint8_t *d_blocks,
                             uint8_t *d_state, void *stream);

/* ---- allocation-free step ------------------------------------------------- */

/* squeeze_step_noalloc -- one tiled step (as squeeze_step with
 * SQUEEZE_STEP_TILED, n_steps = 1) that allocates no memory, for callers
 * that may not call cudaMalloc: code inside an application or framework that
 * owns the whole device-memory budget, and latency-critical code that cannot
 * afford the device-wide synchronisation of cudaMalloc/cudaFree.  The paper
 * has no counterpart; this is an interface of this library only.
 *   s, k, offsets, r   the fractal, validated as in squeeze_create.
 *   birth, survive     9-bit rule masks (B3/S23: 1<<3, (1<<2)|(1<<3)).
 *   d_in, d_out        device buffers of k^r bytes, 16-byte aligned, not
 *                      overlapping; the step reads d_in and writes d_out.
 *   h_status           NULL, or a host int that receives the device status
 *                      (OK / DEVICE_BOUNDS / DEVICE_TIMEOUT); when given, the
 *                      call waits for the step to finish.
 * All scratch (neighbour program, halo tables, per-tile adjacency table and
 * the status word) lives in one fixed 4 MiB device array that every GPU
 * loading the library keeps until exit; a level whose scratch would not fit
 * (the Sierpinski triangle above r = 16, for instance) is rejected with
 * UNSUPPORTED and a message in squeeze_last_cuda_error().  The first call on
 * a device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.  Under
 * the CUDA runtime's lazy module loading (the default since CUDA 12.2) that
 * first call is also what loads the code and the array onto the device, so
 * it takes the array's 4 MiB and the kernels' code memory then, and can fail
 * with a CUDA error when the device is full: an application that will own
 * all device memory makes one call (on a small fractal) at start-up, before
 * it reserves its budget.  Later calls take no device memory.  Every call
 * rewrites the array and clears its status word, so calls that overlap on
 * the GPU (different streams, or threads without ordering) race on it. */
int squeeze_step_noalloc(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                         uint32_t birth, uint32_t survive, const uint8_t *d_in, uint8_t *d_out,
                         int *h_status, void *stream);

/* ---- checkpoint / resume ---------------------------------------------------
 * A run is resumed from (fractal, level, step count, compact state).  These
 * two calls are host code only: the caller copies the state between device
 * and host (the state is caller-owned, like every buffer).  The paper has no
 * counterpart; this is an interface of this library only.  File layout,
 * little-endian: a 64-byte header (magic "SQZSTATE", version 1, header size,
 * s, k, r, dimensions = 2, step, state bytes k^r, FNV-1a 64-bit hash of the
 * state, FNV-1a 64-bit hash of the header with this last word as 0 followed
 * by the padded offsets), the 2k offset bytes zero-padded to a multiple of 8,
 * then the k^r state bytes in compact order.  A single damaged byte anywhere
 * in the file changes one of the two hashes.  The rule and neighbourhood are
 * not stored: they belong to the handle that resumes the run. */

/* squeeze_checkpoint_write -- write h_state (k^r bytes) and `step` to `path`.
 * The fractal is validated as in squeeze_create.  The file is written under
 * a temporary name beside `path` and renamed into place, so readers never see
 * a partial file.  Errors: INVALID_ARG; IO (create, write or rename failed;
 * squeeze_last_cuda_error() holds the reason). */
int squeeze_checkpoint_write(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                             uint64_t step, const uint8_t *h_state, const char *path);

/* squeeze_checkpoint_read -- read a checkpoint of the given fractal and level
 * into h_state (k^r bytes) and *step.  Errors: INVALID_ARG for a bad
 * descriptor or a valid checkpoint of another fractal, offset table or
 * level; IO for a missing or unreadable file, a file that is not a
 * checkpoint, a truncated or over-long file, or a header or state whose hash
 * does not match.  After an error h_state's contents are unspecified and *step is not
 * written. */
int squeeze_checkpoint_read(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                            uint64_t *step, uint8_t *h_state, const char *path);

/* ---- three-dimensional NBB fractals ---------------------------------------
 * The abstract and Sec. 7 name the extension of the compact maps to three
 * dimensions without defining it; this library carries Secs. 3.1-3.4 and 4
 * over to a third axis:
 *   - replicas at distinct offsets tau(beta) = (tau_x, tau_y, tau_z) in
 *     [0, s)^3; a point of the n^3 box (n = s^r) is a cell iff every base-s
 *     digit triple of its coordinates is an offset;
 *   - compact layout: level mu puts its replica id into base-k digit
 *     floor((mu-1)/3) of w_x, w_y or w_z for (mu-1) mod 3 = 0, 1, 2, so
 *     W_x = k^ceil(r/3), W_y = k^floor((r+1)/3), W_z = k^floor(r/3), stored
 *     as omega = (w_z * W_y + w_y) * W_x + w_x; one byte per cell, alive iff
 *     bit 0 is set, k^r bytes per state;
 *   - step: every cell counts its alive fractal neighbours among the offsets
 *     (dx, dy, dz) selected by a 27-bit mask (bit (dz+1)*9 + (dy+1)*3 +
 *     (dx+1); all 26 by default), holes and points off the box dead, and a
 *     27-bit birth/survive rule gives its next state (default B5/S45, Bays'
 *     three-dimensional Life).
 * Conventions (return codes, d_ pointers, streams, device status) are those
 * of the two-dimensional entry points. */
typedef struct squeeze_3d_handle squeeze_3d_handle;

/* squeeze_3d_create -- describe a level-r 3-D NBB fractal.
 *   s        2 <= s <= 8.
 *   k        1 <= k <= min(s^3, 255).
 *   offsets  host array of 3*k bytes: replica beta at (offsets[3*beta],
 *            offsets[3*beta+1], offsets[3*beta+2]), each < s, all distinct.
 *   r        level; requires s^r <= 2^30 and k^r <= 2^40.
 * Errors: INVALID_ARG for any violated bound (checked before any device
 * work); OOM / CUDA when the status word cannot be allocated. */
int squeeze_3d_create(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                      squeeze_3d_handle **out);

/* squeeze_3d_destroy -- synchronise the device and free the handle.  NULL is
 * accepted. */
int squeeze_3d_destroy(squeeze_3d_handle *h);

/* squeeze_3d_info -- k^r cells, the compact extents W_x, W_y, W_z and the
 * side n = s^r.  Any output pointer may be NULL. */
int squeeze_3d_info(const squeeze_3d_handle *h, uint64_t *n_cells, uint64_t *wx, uint64_t *wy,
                    uint64_t *wz, uint64_t *side);

/* squeeze_3d_set_rule -- 27-bit birth/survive masks over the neighbour count
 * 0..26.  Affects steps enqueued after the call. */
int squeeze_3d_set_rule(squeeze_3d_handle *h, uint32_t birth, uint32_t survive);

/* squeeze_3d_set_neighbourhood -- 27-bit offset mask (bit 13, the cell
 * itself, must be clear). */
int squeeze_3d_set_neighbourhood(squeeze_3d_handle *h, uint32_t mask);

/* squeeze_3d_lambda -- compact -> expanded.  d_omega: count uint64 (8-byte
 * aligned); d_xyz (4-byte aligned) receives 3*count int32 (x, y, z),
 * (-1, -1, -1) for an index >= k^r.  A misaligned pointer is INVALID_ARG. */
int squeeze_3d_lambda(const squeeze_3d_handle *h, const uint64_t *d_omega, int32_t *d_xyz,
                      uint64_t count, void *stream);

/* squeeze_3d_nu -- expanded -> compact with hole rejection.  d_xyz: 3*count
 * int32 points (4-byte aligned), any values; d_omega (8-byte aligned)
 * receives the compact index, or UINT64_MAX for a hole or a point off the
 * box.  A misaligned pointer is INVALID_ARG. */
int squeeze_3d_nu(const squeeze_3d_handle *h, const int32_t *d_xyz, uint64_t *d_omega,
                  uint64_t count, void *stream);

/* squeeze_3d_init_bernoulli -- d_state[omega] = 1 iff the top 24 bits of
 * SplitMix64 output number omega of the stream seeded with `seed` are below
 * p_q24 (<= 2^24), else 0. */
int squeeze_3d_init_bernoulli(const squeeze_3d_handle *h, uint8_t *d_state, uint64_t seed,
                              uint32_t p_q24, void *stream);

/* squeeze_3d_step -- n_steps steps: the bit-sliced tile kernel where it
 * applies (squeeze_3d_set_tiled_level), else one thread per compact cell:
 * lambda's digits, each neighbour by the carry walk of nu from the cell's own
 * digits, the rule into the other buffer.  Result in d_buf0 when n_steps is even,
 * d_buf1 when odd; the buffers (k^r bytes each) must differ.  A neighbour
 * index past the state (impossible for a valid handle) is skipped and
 * latches DEVICE_BOUNDS. */
int squeeze_3d_step(squeeze_3d_handle *h, uint8_t *d_buf0, uint8_t *d_buf1, uint64_t n_steps,
                    void *stream);

/* squeeze_3d_set_tiled_level -- which kernel squeeze_3d_step runs.  The
 * bit-sliced tile kernel (level-L sub-replicas of k^L cells as tiles, a
 * host-built 26-neighbour program per level, the adjacent tile in each of the
 * 26 directions from a per-handle table, 32 tiles per CTA bit-sliced into
 * 32-bit words) takes levels whose tile rows hold 8 or 16 cells
 * (k^ceil(L/3) = 8 or 16), with W_x a multiple of 16 and 16-byte aligned
 * buffers; otherwise (the Menger sponge, say) the per-cell kernel runs.
 *   level 0      the per-cell kernel always;
 *   0 < L <= r   the tile kernel at level L (UNSUPPORTED if it cannot take L).
 * By default the largest level with at most 1024 slot words is used.  The
 * results are the same bit for bit. */
int squeeze_3d_set_tiled_level(squeeze_3d_handle *h, uint32_t level);

/* squeeze_3d_tiled_level -- the level the tile kernel runs at (aligned
 * buffers), or 0 when squeeze_3d_step runs the per-cell kernel. */
int squeeze_3d_tiled_level(const squeeze_3d_handle *h);

/* squeeze_3d_device_status -- as squeeze_device_status, for a 3-D handle. */
int squeeze_3d_device_status(squeeze_3d_handle *h, int *status);

/* ---- diagnostics ---------------------------------------------------------- */

/* squeeze_device_status -- synchronise the device, then read and clear the
 * handle's device status word: *status = SQUEEZE_OK, DEVICE_BOUNDS,
 * DEVICE_TIMEOUT or DEVICE_UNSAFE.  DEVICE_TIMEOUT: a wait of the tiled
 * kernel on its bulk copies gave up; that CTA stopped loading, the launch's
 * output is not valid, and the copy it waited for was accounted for before
 * the kernel ended, so later launches are safe.  DEVICE_UNSAFE: the copy a
 * CTA gave up on had still not landed after a second wait of the same limit;
 * it may still write into shared memory that a later launch owns, so the
 * context should be discarded.  Returns CUDA if the synchronisation itself
 * failed. */
int squeeze_device_status(squeeze_handle *h, int *status);

/* squeeze_set_wait_limit -- how long a device-side wait of this handle's
 * tiled and batched steps spins before it gives up with DEVICE_TIMEOUT:
 * ns in [1000, 10^10] nanoseconds of %globaltimer, or 0 for the default of
 * 2 s.  INVALID_ARG otherwise.  A batch reads the limit of each item's handle
 * when it is created. */
int squeeze_set_wait_limit(squeeze_handle *h, uint64_t ns);

/* squeeze_set_fault_injection -- test hook for the device error paths:
 * flags = 0 (off) or SQUEEZE_FAULT_WITHHOLD_LOADS, under which the tiled step
 * issues none of its bulk loads, so that its first wait runs out after the
 * wait limit, every CTA abandons its work, and the launch ends with
 * DEVICE_TIMEOUT in the status word (nothing is left in flight: no copy was
 * issued).  The output buffer then holds garbage in place of the step's
 * result.  INVALID_ARG for unknown flags. */
int squeeze_set_fault_injection(squeeze_handle *h, uint32_t flags);

/* squeeze_status_string -- static text for a status code. */
const char *squeeze_status_string(int status);

/* squeeze_last_cuda_error -- text of the last CUDA error this thread saw in
 * the library ("" when none). */
const char *squeeze_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SQUEEZE_H */
