/*
 * nbb3d_oracle.c -- plain CPU oracle for three-dimensional NBB fractals.
 *
 * TEST INFRASTRUCTURE, not part of the product.  Only the test suite and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code,
 * header, table or helper with the CUDA library; it is linked into the same
 * oracle library as squeeze_oracle.c and uses that file's SplitMix64.
 *
 * Paper: Quezada, Navarro, Hitschfeld, Bustos, "Squeeze: Efficient Compact
 * Fractals for Tensor Core GPUs" (arXiv 2201.00613).  The abstract and the
 * conclusions (Sec. 7) say that the compact maps extend to three dimensions;
 * the paper gives no definition, so this file follows reading R15, which
 * carries the two-dimensional definitions of Secs. 3.1-3.4 and 4 over to a
 * third axis:
 *   R15a  A 3-D NBB fractal has k replicas per level at distinct offsets
 *         tau(beta) = (tau_x, tau_y, tau_z) in [0, s)^3.  A point of the
 *         n x n x n box (n = s^r) is a level-r cell iff, at every level
 *         mu = 1..r, its base-s digit triple at position mu-1 is an offset.
 *   R15b  Compact layout: the levels cycle over the compact axes x, y, z.
 *         Level mu puts its replica id beta_mu into the base-k digit at
 *         position floor((mu-1)/3) of w_x, w_y or w_z for (mu-1) mod 3 =
 *         0, 1, 2.  So W_x = k^ceil(r/3), W_y = k^floor((r+1)/3),
 *         W_z = k^floor(r/3), and omega = (w_z * W_y + w_y) * W_x + w_x.
 *   R15c  lambda(omega) = sum over mu of tau(beta_mu) * s^(mu-1) on each
 *         axis; nu is its inverse, rejecting a point whose digit triple at
 *         some level is not an offset (a hole) or that lies off the box.
 *   R15d  Step: an outer-totalistic rule over the neighbourhood mask (bit
 *         (dz+1)*9 + (dy+1)*3 + (dx+1) selects offset (dx, dy, dz); all 26 by
 *         default); birth and survive are 27-bit masks over the count of
 *         alive fractal neighbours; holes and points off the box are dead;
 *         synchronous update into a second buffer.
 *   R15e  Initial state: the cell at compact index omega is alive iff the
 *         top 24 bits of SplitMix64 output number omega (seeded with `seed`)
 *         are below p_q24.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

uint64_t orc_splitmix64(uint64_t seed, uint64_t i);   /* squeeze_oracle.c */

static uint64_t o3_pow(uint64_t b, uint32_t e) {
    uint64_t p = 1;
    while (e--) p *= b;
    return p;
}

/* Compact extents (R15b): count the levels that land on each axis. */
void o3_extents(uint32_t k, uint32_t r, uint64_t *wx, uint64_t *wy, uint64_t *wz) {
    uint32_t levels[3] = {0, 0, 0};
    for (uint32_t mu = 1; mu <= r; ++mu) levels[(mu - 1) % 3]++;
    *wx = o3_pow(k, levels[0]);
    *wy = o3_pow(k, levels[1]);
    *wz = o3_pow(k, levels[2]);
}

/* Replica id of a digit triple: the index beta with tau(beta) equal to it,
 * found by a plain search over the offset table; -1 for a hole. */
static int o3_replica(uint32_t k, const uint8_t *tau, uint32_t dx, uint32_t dy, uint32_t dz) {
    for (uint32_t b = 0; b < k; ++b)
        if (tau[3 * b] == dx && tau[3 * b + 1] == dy && tau[3 * b + 2] == dz) return (int)b;
    return -1;
}

/* Membership (R15a). */
int o3_member(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
              int64_t x, int64_t y, int64_t z) {
    int64_t n = (int64_t)o3_pow(s, r);
    if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n) return 0;
    for (uint32_t mu = 1; mu <= r; ++mu) {
        int64_t p = (int64_t)o3_pow(s, mu - 1);
        uint32_t dx = (uint32_t)((x / p) % s);
        uint32_t dy = (uint32_t)((y / p) % s);
        uint32_t dz = (uint32_t)((z / p) % s);
        if (o3_replica(k, tau, dx, dy, dz) < 0) return 0;
    }
    return 1;
}

/* n^3 membership box, index (z * n + y) * n + x. */
void o3_member_grid(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r, uint8_t *out) {
    int64_t n = (int64_t)o3_pow(s, r);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < n; ++z)
        for (int64_t y = 0; y < n; ++y)
            for (int64_t x = 0; x < n; ++x)
                out[(z * n + y) * n + x] = (uint8_t)o3_member(s, k, tau, r, x, y, z);
}

/* lambda (R15b, R15c): compact index -> (x, y, z); -1s past the last cell. */
static void o3_lambda(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r, uint64_t omega,
                      int64_t *xyz) {
    uint64_t Wx, Wy, Wz;
    o3_extents(k, r, &Wx, &Wy, &Wz);
    if (omega >= Wx * Wy * Wz) {
        xyz[0] = xyz[1] = xyz[2] = -1;
        return;
    }
    uint64_t w[3];
    w[0] = omega % Wx;
    w[1] = (omega / Wx) % Wy;
    w[2] = omega / Wx / Wy;
    int64_t acc[3] = {0, 0, 0};
    for (uint32_t mu = 1; mu <= r; ++mu) {
        uint32_t axis = (mu - 1) % 3, pos = (mu - 1) / 3;
        uint32_t beta = (uint32_t)((w[axis] / o3_pow(k, pos)) % k);
        int64_t scale = (int64_t)o3_pow(s, mu - 1);
        for (int a = 0; a < 3; ++a) acc[a] += (int64_t)tau[3 * beta + a] * scale;
    }
    xyz[0] = acc[0];
    xyz[1] = acc[1];
    xyz[2] = acc[2];
}

/* nu (R15c): (x, y, z) -> compact index, UINT64_MAX for a hole or off the box. */
static uint64_t o3_nu(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                      int64_t x, int64_t y, int64_t z) {
    int64_t n = (int64_t)o3_pow(s, r);
    if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n) return UINT64_MAX;
    uint64_t Wx, Wy, Wz;
    o3_extents(k, r, &Wx, &Wy, &Wz);
    uint64_t w[3] = {0, 0, 0};
    for (uint32_t mu = 1; mu <= r; ++mu) {
        int64_t p = (int64_t)o3_pow(s, mu - 1);
        int beta = o3_replica(k, tau, (uint32_t)((x / p) % s), (uint32_t)((y / p) % s),
                              (uint32_t)((z / p) % s));
        if (beta < 0) return UINT64_MAX;
        w[(mu - 1) % 3] += (uint64_t)beta * o3_pow(k, (mu - 1) / 3);
    }
    return (w[2] * Wy + w[1]) * Wx + w[0];
}

void o3_lambda_many(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                    const uint64_t *omega, int64_t *xyz, int64_t count) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) o3_lambda(s, k, tau, r, omega[i], xyz + 3 * i);
}

void o3_nu_many(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                const int64_t *xyz, uint64_t *omega, int64_t count) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i)
        omega[i] = o3_nu(s, k, tau, r, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
}

/* Scatter a compact state (k^r bytes) into a zeroed n^3 box through lambda. */
void o3_compact_to_box(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                       const uint8_t *compact, uint8_t *box) {
    int64_t n = (int64_t)o3_pow(s, r), cells = (int64_t)o3_pow(k, r);
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < cells; ++w) {
        int64_t p[3];
        o3_lambda(s, k, tau, r, (uint64_t)w, p);
        box[(p[2] * n + p[1]) * n + p[0]] = compact[w];
    }
}

/* Gather the fractal cells of an n^3 box into compact order. */
void o3_box_to_compact(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r,
                       const uint8_t *box, uint8_t *compact) {
    int64_t n = (int64_t)o3_pow(s, r), cells = (int64_t)o3_pow(k, r);
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < cells; ++w) {
        int64_t p[3];
        o3_lambda(s, k, tau, r, (uint64_t)w, p);
        compact[w] = box[(p[2] * n + p[1]) * n + p[0]];
    }
}

static int o3_in_nbhd(uint32_t mask, int dx, int dy, int dz) {
    return (int)((mask >> ((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1))) & 1u);
}

/* One synchronous step of the box automaton (R15d): every fractal cell
 * counts its alive fractal neighbours in the mask; holes stay 0. */
void o3_box_step(int64_t n, const uint8_t *member, const uint8_t *in, uint8_t *out,
                 uint32_t birth, uint32_t survive, uint32_t nbhd) {
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < n; ++z)
        for (int64_t y = 0; y < n; ++y)
            for (int64_t x = 0; x < n; ++x) {
                int64_t p = (z * n + y) * n + x;
                if (!member[p]) {
                    out[p] = 0;
                    continue;
                }
                uint32_t c = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if ((dx == 0 && dy == 0 && dz == 0) || !o3_in_nbhd(nbhd, dx, dy, dz))
                                continue;
                            int64_t qx = x + dx, qy = y + dy, qz = z + dz;
                            if (qx < 0 || qy < 0 || qz < 0 || qx >= n || qy >= n || qz >= n)
                                continue;
                            int64_t q = (qz * n + qy) * n + qx;
                            if (member[q] && (in[q] & 1u)) ++c;
                        }
                uint32_t mask = (in[p] & 1u) ? survive : birth;
                out[p] = (uint8_t)((mask >> c) & 1u);
            }
}

/* `steps` box steps; the result is left in a (b is scratch). */
void o3_box_run(int64_t n, const uint8_t *member, uint8_t *a, uint8_t *b, int64_t steps,
                uint32_t birth, uint32_t survive, uint32_t nbhd) {
    size_t bytes = (size_t)(n * n * n);
    for (int64_t t = 0; t < steps; ++t) {
        o3_box_step(n, member, a, b, birth, survive, nbhd);
        memcpy(a, b, bytes);
    }
}

/* Initial compact state (R15e). */
void o3_init_compact(uint64_t seed, uint32_t p_q24, int64_t cells, uint8_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < cells; ++w)
        out[w] = (uint8_t)((orc_splitmix64(seed, (uint64_t)w) >> 40) < p_q24);
}

/* Light-cone sampler: the state after T steps at each sample cell (x, y, z),
 * from the R15e start.  A (2T+1)^3 window around the sample is filled (its
 * fractal cells from nu and R15e), and T box steps run on it with everything
 * beyond the window dead; after step t only the cells within Chebyshev
 * distance T-t of the centre are still exact, so only those are updated. */
void o3_lightcone(uint32_t s, uint32_t k, const uint8_t *tau, uint32_t r, uint64_t seed,
                  uint32_t p_q24, int64_t T, uint32_t birth, uint32_t survive, uint32_t nbhd,
                  const int64_t *xyz, int64_t count, uint8_t *out) {
    int64_t w = 2 * T + 1, vol = w * w * w;
#pragma omp parallel
    {
        uint8_t *mem = (uint8_t *)malloc((size_t)vol);
        uint8_t *a = (uint8_t *)malloc((size_t)vol);
        uint8_t *b = (uint8_t *)malloc((size_t)vol);
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < count; ++i) {
            int64_t cx = xyz[3 * i], cy = xyz[3 * i + 1], cz = xyz[3 * i + 2];
            for (int64_t l = 0; l < w; ++l)
                for (int64_t j = 0; j < w; ++j)
                    for (int64_t q = 0; q < w; ++q) {
                        int64_t x = cx - T + q, y = cy - T + j, z = cz - T + l;
                        int64_t p = (l * w + j) * w + q;
                        uint64_t om = o3_nu(s, k, tau, r, x, y, z);
                        mem[p] = om != UINT64_MAX;
                        a[p] = mem[p] ? (uint8_t)((orc_splitmix64(seed, om) >> 40) < p_q24) : 0;
                    }
            memcpy(b, a, (size_t)vol);
            for (int64_t t = 1; t <= T; ++t) {
                int64_t lo = t, hi = w - 1 - t;
                for (int64_t l = lo; l <= hi; ++l)
                    for (int64_t j = lo; j <= hi; ++j)
                        for (int64_t q = lo; q <= hi; ++q) {
                            int64_t p = (l * w + j) * w + q;
                            if (!mem[p]) {
                                b[p] = 0;
                                continue;
                            }
                            uint32_t c = 0;
                            for (int dz = -1; dz <= 1; ++dz)
                                for (int dy = -1; dy <= 1; ++dy)
                                    for (int dx = -1; dx <= 1; ++dx) {
                                        if ((dx == 0 && dy == 0 && dz == 0) ||
                                            !o3_in_nbhd(nbhd, dx, dy, dz))
                                            continue;
                                        int64_t pq = ((l + dz) * w + (j + dy)) * w + (q + dx);
                                        if (mem[pq] && a[pq]) ++c;
                                    }
                            uint32_t mask = a[p] ? survive : birth;
                            b[p] = (uint8_t)((mask >> c) & 1u);
                        }
                uint8_t *tmp = a;
                a = b;
                b = tmp;
            }
            out[i] = a[(T * w + T) * w + T];
        }
        free(mem);
        free(a);
        free(b);
    }
}
