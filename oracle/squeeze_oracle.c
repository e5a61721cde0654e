/*
 * squeeze_oracle.c -- plain CPU oracle for the compact-fractal cellular automaton.
 *
 * TEST INFRASTRUCTURE, not part of the product.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load this file's library.
 * It shares no code, header, table or helper with the CUDA library: every
 * quantity below is recomputed from the paper's definitions, in the paper's
 * order, with no blocking or fusion.  It is deliberately slow.
 *
 * Paper: Quezada, Navarro, Hitschfeld, Bustos, "Squeeze: Efficient Compact
 * Fractals for Tensor Core GPUs" (arXiv 2201.00613).
 *
 * Readings of passages that are garbled or at odds with each other (each one is
 * also listed with its reason in the design notes):
 *   R1 (Eq. theta): the printed digit  floor((w mod s^mu) / s^mu)  is always 0;
 *       it is read as the base-s digit at position mu-1:
 *       theta_mu = floor((w mod s^mu) / s^(mu-1)).
 *   R2 (Eq. f): the printed filter f_x(mu) = (mu-1) mod 2 sends even levels to
 *       x, while Eq. beta (and the compaction rule of Sec. 3.1) send odd levels
 *       to x.  nu is defined as the inverse of lambda (Sec. 3.4), so the filter
 *       is read as f_x(mu) = mu mod 2, f_y(mu) = (mu-1) mod 2.
 *   R3 (Eq. siertx): the Sierpinski weight 3^((mu-1)/2) lacks the floor of
 *       Eq. t; it is read as k^floor((mu-1)/2).
 *   R4 (Sec. 3.4): H_nu is "a table of size k" keyed by theta in [0,s)^2; it is
 *       read as an s*s table whose non-replica entries mark a hole.
 *   R5 (Sec. 3.1): the compact rectangle has W = k^ceil(r/2) columns (the odd
 *       levels, x) and H = k^floor(r/2) rows; storage is row-major,
 *       linear index = w_y * W + w_x.
 *   R6 (Sec. 4): the "adapted" Life rule is B3/S23 counted over fractal
 *       neighbours only; cells outside the box and holes are dead; no wrap;
 *       synchronous update into a second buffer.  Other birth/survive masks
 *       are accepted as 9-bit masks over the neighbour count.
 *   R10 (silent): one byte per cell; a cell is alive iff bit 0 of its byte
 *       is set.  States written here are 0 or 1.
 *   R7 (initial states): cell (x, y) is alive iff the top 24 bits of output
 *       number (y * 2^32 + x) of a SplitMix64 stream seeded with `seed` are
 *       below p_q24 (SplitMix64: Steele, Lea, Flood, OOPSLA 2014).
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static uint64_t orc_ipow(uint64_t b, uint32_t e) {
    uint64_t p = 1;
    while (e--) p *= b;
    return p;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* NBB membership (Sec. 1 and Sec. 3: replicas only translate, never overlap).
 * (x, y) is a cell of the level-r fractal iff, for every level mu = 1..r, the
 * base-s digit pair of (x, y) at position mu-1 equals one of the k replica
 * offsets tau(beta).  Anything outside [0, s^r)^2 is not a cell.            */
int orc_member(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r, int64_t x, int64_t y) {
    int64_t n = (int64_t)orc_ipow(s, r);
    if (x < 0 || y < 0 || x >= n || y >= n) return 0;
    for (uint32_t mu = 1; mu <= r; ++mu) {
        int64_t p = (int64_t)orc_ipow(s, mu - 1);
        uint32_t dx = (uint32_t)((x / p) % s);
        uint32_t dy = (uint32_t)((y / p) % s);
        int found = 0;
        for (uint32_t b = 0; b < k; ++b)
            if (tau[2 * b] == dx && tau[2 * b + 1] == dy) found = 1;
        if (!found) return 0;
    }
    return 1;
}

/* Membership of every cell of the n x n box, row-major (y * n + x). */
void orc_member_grid(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r, uint8_t *out) {
    int64_t n = (int64_t)orc_ipow(s, r);
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x)
            out[y * n + x] = (uint8_t)orc_member(s, k, tau, r, x, y);
}

/* ------------------------------------------------------------------------- */
/* lambda: compact -> expanded (Sec. 3.3, Eqs. lambda, Delta_mu, tau, beta).
 *   beta_mu = floor((w_x (mu mod 2) + w_y ((mu+1) mod 2)) / k^(ceil(mu/2)-1)) mod k
 *   lambda(w) = sum_{mu=1..r} tau(beta_mu) * s^(mu-1)                         */
void orc_lambda(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                uint64_t wx, uint64_t wy, int64_t *x, int64_t *y) {
    int64_t X = 0, Y = 0;
    for (uint32_t mu = 1; mu <= r; ++mu) {
        uint64_t source = wx * (mu % 2) + wy * ((mu + 1) % 2);
        uint32_t ceil_half = (mu + 1) / 2;
        uint64_t beta = (source / orc_ipow(k, ceil_half - 1)) % k;
        int64_t scale = (int64_t)orc_ipow(s, mu - 1);
        X += (int64_t)tau[2 * beta] * scale;
        Y += (int64_t)tau[2 * beta + 1] * scale;
    }
    *x = X;
    *y = Y;
}

/* ------------------------------------------------------------------------- */
/* nu: expanded -> compact (Sec. 3.4, Eqs. theta, t, f, nux, nuy; readings
 * R1, R2, R4).  Returns 1 and writes (w_x, w_y) for a fractal cell, returns 0
 * for a hole or a point outside the box.
 *   theta_mu = (floor((x mod s^mu)/s^(mu-1)), floor((y mod s^mu)/s^(mu-1)))
 *   Delta^nu_mu = k^floor((mu-1)/2)
 *   nu_x = sum Delta^nu_mu H_nu[theta_mu] f_x(mu),  nu_y likewise with f_y. */
int orc_nu(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
           int64_t x, int64_t y, uint64_t *wx, uint64_t *wy) {
    int64_t n = (int64_t)orc_ipow(s, r);
    if (x < 0 || y < 0 || x >= n || y >= n) return 0;
    int hnu[64 * 64];
    for (uint32_t i = 0; i < s * s; ++i) hnu[i] = -1;
    for (uint32_t b = 0; b < k; ++b) hnu[tau[2 * b + 1] * s + tau[2 * b]] = (int)b;
    uint64_t nx = 0, ny = 0;
    for (uint32_t mu = 1; mu <= r; ++mu) {
        int64_t lo = (int64_t)orc_ipow(s, mu - 1);
        int64_t hi = lo * (int64_t)s;
        uint32_t theta_x = (uint32_t)((x % hi) / lo);
        uint32_t theta_y = (uint32_t)((y % hi) / lo);
        int h = hnu[theta_y * s + theta_x];
        if (h < 0) return 0;
        uint64_t delta = orc_ipow(k, (mu - 1) / 2);
        uint64_t fx = mu % 2, fy = (mu - 1) % 2;
        nx += delta * (uint64_t)h * fx;
        ny += delta * (uint64_t)h * fy;
    }
    *wx = nx;
    *wy = ny;
    return 1;
}

/* Element-wise lambda over `count` linear compact indices (row-major, R5).
 * Out-of-range indices give (-1, -1). */
void orc_lambda_many(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                     const uint64_t *omega, int64_t *xy, int64_t count) {
    uint64_t W = orc_ipow(k, (r + 1) / 2), cells = orc_ipow(k, r);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        if (omega[i] >= cells) { xy[2 * i] = -1; xy[2 * i + 1] = -1; continue; }
        orc_lambda(s, k, tau, r, omega[i] % W, omega[i] / W, &xy[2 * i], &xy[2 * i + 1]);
    }
}

/* Element-wise nu over `count` expanded points; holes and outside -> UINT64_MAX. */
void orc_nu_many(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                 const int64_t *xy, uint64_t *omega, int64_t count) {
    uint64_t W = orc_ipow(k, (r + 1) / 2);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        uint64_t wx, wy;
        if (orc_nu(s, k, tau, r, xy[2 * i], xy[2 * i + 1], &wx, &wy))
            omega[i] = wy * W + wx;
        else
            omega[i] = UINT64_MAX;
    }
}

/* ------------------------------------------------------------------------- */
/* Canonical enumeration: copy a compact buffer (W x H row-major, R5) into the
 * n x n box at lambda(w), and back.  Cells of the box that no w reaches keep
 * the value they had (callers pass a zeroed box).                            */
void orc_compact_to_box(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                        const uint8_t *compact, uint8_t *box) {
    uint64_t W = orc_ipow(k, (r + 1) / 2), H = orc_ipow(k, r / 2);
    int64_t n = (int64_t)orc_ipow(s, r);
#pragma omp parallel for schedule(static)
    for (int64_t wy = 0; wy < (int64_t)H; ++wy)
        for (uint64_t wx = 0; wx < W; ++wx) {
            int64_t x, y;
            orc_lambda(s, k, tau, r, wx, (uint64_t)wy, &x, &y);
            box[y * n + x] = compact[(uint64_t)wy * W + wx];
        }
}

void orc_box_to_compact(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                        const uint8_t *box, uint8_t *compact) {
    uint64_t W = orc_ipow(k, (r + 1) / 2), H = orc_ipow(k, r / 2);
    int64_t n = (int64_t)orc_ipow(s, r);
#pragma omp parallel for schedule(static)
    for (int64_t wy = 0; wy < (int64_t)H; ++wy)
        for (uint64_t wx = 0; wx < W; ++wx) {
            int64_t x, y;
            orc_lambda(s, k, tau, r, wx, (uint64_t)wy, &x, &y);
            compact[(uint64_t)wy * W + wx] = box[y * n + x];
        }
}

/* ------------------------------------------------------------------------- */
/* Bounding-box cellular-automaton step (Sec. 4; readings R6, R10).  `member`
 * marks the fractal cells of the n x n box.  For a fractal cell p with c alive
 * fractal Moore neighbours: next = alive ? bit c of survive : bit c of birth.
 * Non-fractal cells are written 0.                                          */
void orc_box_step(int64_t n, const uint8_t *member, const uint8_t *in, uint8_t *out,
                  uint32_t birth, uint32_t survive) {
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x) {
            int64_t p = y * n + x;
            if (!member[p]) { out[p] = 0; continue; }
            uint32_t c = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    int64_t qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= n || qy >= n) continue;
                    int64_t q = qy * n + qx;
                    if (member[q] && (in[q] & 1u)) ++c;
                }
            uint32_t mask = (in[p] & 1u) ? survive : birth;
            out[p] = (uint8_t)((mask >> c) & 1u);
        }
}

/* `steps` synchronous steps, ping-ponging between `a` and `b`; the result is
 * left in `a` (copied back when steps is odd). */
void orc_box_run(int64_t n, const uint8_t *member, uint8_t *a, uint8_t *b, int64_t steps,
                 uint32_t birth, uint32_t survive) {
    for (int64_t t = 0; t < steps; ++t) {
        orc_box_step(n, member, a, b, birth, survive);
        uint8_t *tmp = a; a = b; b = tmp;
    }
    if (steps % 2) memcpy(b, a, (size_t)(n * n));
}

/* ------------------------------------------------------------------------- */
/* Other neighbourhoods and a PDE on the fractal (Sec. 1 names stencil
 * simulations, cellular automata and PDE solvers as the uses of the compact
 * maps).  A neighbourhood is a 9-bit mask over the 3 x 3 block: bit
 * (dy + 1) * 3 + (dx + 1) selects offset (dx, dy); bit 4 (the cell itself)
 * is ignored.  Moore is 0x1EF, von Neumann 0xAA.                            */

static int orc_in_nbhd(uint32_t nbhd, int dx, int dy) {
    return (dx || dy) && ((nbhd >> ((dy + 1) * 3 + (dx + 1))) & 1u);
}

/* One outer-totalistic step counting only the fractal neighbours in `nbhd`. */
void orc_box_step_nbhd(int64_t n, const uint8_t *member, const uint8_t *in, uint8_t *out,
                       uint32_t birth, uint32_t survive, uint32_t nbhd) {
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x) {
            int64_t p = y * n + x;
            if (!member[p]) { out[p] = 0; continue; }
            uint32_t c = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!orc_in_nbhd(nbhd, dx, dy)) continue;
                    int64_t qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= n || qy >= n) continue;
                    int64_t q = qy * n + qx;
                    if (member[q] && (in[q] & 1u)) ++c;
                }
            uint32_t mask = (in[p] & 1u) ? survive : birth;
            out[p] = (uint8_t)((mask >> c) & 1u);
        }
}

void orc_box_run_nbhd(int64_t n, const uint8_t *member, uint8_t *a, uint8_t *b, int64_t steps,
                      uint32_t birth, uint32_t survive, uint32_t nbhd) {
    for (int64_t t = 0; t < steps; ++t) {
        orc_box_step_nbhd(n, member, a, b, birth, survive, nbhd);
        uint8_t *tmp = a; a = b; b = tmp;
    }
    if (steps % 2) memcpy(b, a, (size_t)(n * n));
}

/* Explicit Euler steps of the heat equation on the fractal graph, in fp64:
 * u'(p) = u(p) + alpha * sum over fractal neighbours q of p in `nbhd` of
 * (u(q) - u(p)); cells off the fractal stay 0.  Result left in `a`.        */
void orc_heat_run(int64_t n, const uint8_t *member, double *a, double *b, int64_t steps,
                  double alpha, uint32_t nbhd) {
    for (int64_t t = 0; t < steps; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < n; ++y)
            for (int64_t x = 0; x < n; ++x) {
                int64_t p = y * n + x;
                if (!member[p]) { b[p] = 0.0; continue; }
                double flow = 0.0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!orc_in_nbhd(nbhd, dx, dy)) continue;
                        int64_t qx = x + dx, qy = y + dy;
                        if (qx < 0 || qy < 0 || qx >= n || qy >= n) continue;
                        int64_t q = qy * n + qx;
                        if (member[q]) flow += a[q] - a[p];
                    }
                b[p] = a[p] + alpha * flow;
            }
        double *tmp = a; a = b; b = tmp;
    }
    if (steps % 2) memcpy(b, a, (size_t)(n * n) * sizeof(double));
}

/* ------------------------------------------------------------------------- */
/* Ising spins on the fractal graph (Sec. 1 names spin-model simulations):
 * spin +1 where bit 0 is set, -1 otherwise, coupling J = 1 between fractal
 * neighbours of the mask (which must join only cells of opposite parity of
 * x + y, e.g. von Neumann).  One sweep is two half-sweeps, cells with
 * (x + y) even first, then odd.  Half-sweep number t (t = 0, 1, ... counted
 * from the first sweep of the call) draws from the SplitMix64 stream seeded
 * with d_t = splitmix64(seed, t); cell (x, y) takes output number
 * y * 2^32 + x of that stream.  With h the sum of the neighbour spins and
 * dE = 2 * s * h, the spin flips iff dE <= 0 or (draw >> 40) < floor(exp(-dE
 * / T) * 2^24) (Metropolis acceptance in 24-bit fixed point).              */
static uint64_t orc_splitmix64_local(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void orc_ising_run(int64_t n, const uint8_t *member, uint8_t *box, int64_t sweeps,
                   uint64_t seed, double temperature, uint32_t nbhd) {
    /* acceptance thresholds for dE = 2, 4, ..., 16 (index dE / 2) */
    uint64_t thr[9];
    thr[0] = 1ull << 24;
    for (int e = 1; e <= 8; ++e) {
        double a = temperature > 0.0 ? exp(-(2.0 * e) / temperature) : 0.0;
        thr[e] = (uint64_t)floor(a * 16777216.0);
    }
    for (int64_t t = 0; t < 2 * sweeps; ++t) {
        const int64_t parity = t & 1;
        const uint64_t d = orc_splitmix64_local(seed, (uint64_t)t);
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < n; ++y)
            for (int64_t x = (y + parity) & 1; x < n; x += 2) {
                int64_t p = y * n + x;
                if (!member[p]) continue;
                int h = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!orc_in_nbhd(nbhd, dx, dy)) continue;
                        int64_t qx = x + dx, qy = y + dy;
                        if (qx < 0 || qy < 0 || qx >= n || qy >= n) continue;
                        int64_t q = qy * n + qx;
                        if (member[q]) h += (box[q] & 1u) ? 1 : -1;
                    }
                const int sp = (box[p] & 1u) ? 1 : -1;
                const int e2 = sp * h;                  /* dE / 2 */
                int flip = e2 <= 0;
                if (!flip) {
                    uint64_t draw = orc_splitmix64_local(d, ((uint64_t)y << 32) | (uint64_t)x);
                    flip = (draw >> 40) < thr[e2];
                }
                if (flip) box[p] = (uint8_t)((box[p] & 1u) ? 0 : 1);
            }
    }
}

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the stream seeded with `seed`
 * returns, as its output number i (i = 0, 1, ...), mix(seed + (i+1) * gamma)
 * with gamma = 0x9E3779B97F4A7C15 and mix the variant-13 finaliser.          */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Initial state of cell (x, y) (reading R7). */
static uint8_t orc_alive0(uint64_t seed, uint32_t p_q24, int64_t x, int64_t y) {
    uint64_t key = ((uint64_t)y << 32) | (uint64_t)x;
    return (uint8_t)((orc_splitmix64(seed, key) >> 40) < p_q24);
}

/* Bernoulli initial state over the box: fractal cells from R7, others 0. */
void orc_box_init(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                  uint64_t seed, uint32_t p_q24, uint8_t *box) {
    int64_t n = (int64_t)orc_ipow(s, r);
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x)
            box[y * n + x] = orc_member(s, k, tau, r, x, y) ? orc_alive0(seed, p_q24, x, y) : 0;
}

/* ------------------------------------------------------------------------- */
/* Light-cone sampler.  The state of cell p after T synchronous steps depends
 * only on the initial states within Chebyshev distance T of p.  For each
 * sample (x, y) a (2T+1)^2 window centred on it is filled from R7 (fractal
 * cells only), then T box steps are run on the window, treating everything
 * beyond the window as dead; after step t only cells within distance T-t of
 * the centre are still exact, so only those are updated.  The centre after T
 * steps is returned.  Samples must be fractal cells.                          */
void orc_lightcone(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                   uint64_t seed, uint32_t p_q24, int64_t T, uint32_t birth, uint32_t survive,
                   const int64_t *xy, int64_t count, uint8_t *out) {
    int64_t w = 2 * T + 1;
#pragma omp parallel
    {
        uint8_t *mem = (uint8_t *)malloc((size_t)(w * w));
        uint8_t *a = (uint8_t *)malloc((size_t)(w * w));
        uint8_t *b = (uint8_t *)malloc((size_t)(w * w));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < count; ++i) {
            int64_t cx = xy[2 * i], cy = xy[2 * i + 1];
            for (int64_t j = 0; j < w; ++j)
                for (int64_t q = 0; q < w; ++q) {
                    int64_t x = cx - T + q, y = cy - T + j;
                    uint8_t m = (uint8_t)orc_member(s, k, tau, r, x, y);
                    mem[j * w + q] = m;
                    a[j * w + q] = m ? orc_alive0(seed, p_q24, x, y) : 0;
                }
            memcpy(b, a, (size_t)(w * w));
            for (int64_t t = 1; t <= T; ++t) {
                int64_t lo = t, hi = w - 1 - t;  /* cells still exact after step t */
                for (int64_t j = lo; j <= hi; ++j)
                    for (int64_t q = lo; q <= hi; ++q) {
                        int64_t p = j * w + q;
                        if (!mem[p]) { b[p] = 0; continue; }
                        uint32_t c = 0;
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                if (dx == 0 && dy == 0) continue;
                                int64_t pq = (j + dy) * w + (q + dx);
                                if (mem[pq] && a[pq]) ++c;
                            }
                        uint32_t mask = a[p] ? survive : birth;
                        b[p] = (uint8_t)((mask >> c) & 1u);
                    }
                uint8_t *tmp = a; a = b; b = tmp;
            }
            out[i] = a[T * w + T];
        }
        free(mem);
        free(a);
        free(b);
    }
}
