// nbb3d.cuh -- three-dimensional NBB fractals in compact form: descriptor,
// lambda, nu and the neighbour walk, per cell.
//
// The paper (arXiv 2201.00613) names the extension of the compact maps to
// three dimensions (abstract, Sec. 7) without defining it.  This library
// carries Secs. 3.1-3.4 over to a third axis: replica offsets
// tau(beta) in [0, s)^3; a point is a level-r cell iff every base-s digit
// triple of its coordinates is an offset; level mu puts its replica id into
// base-k digit floor((mu-1)/3) of the compact coordinate w_x, w_y or w_z for
// (mu-1) mod 3 = 0, 1, 2, so the compact box has W_x = k^ceil(r/3),
// W_y = k^floor((r+1)/3), W_z = k^floor(r/3) and omega = (w_z W_y + w_y) W_x
// + w_x.  The functions are host-callable as well, so that their index
// arithmetic can be checked on the CPU.
#pragma once

#include "squeeze_internal.cuh"

namespace sq3 {

using sq::FastDiv;
using sq::fdiv;

constexpr int kMaxS = 8;                 // H_nu has at most 8^3 = 512 entries
constexpr int kMaxK = 255;
constexpr uint8_t kHole = 0xFF;
constexpr uint32_t kMoore26 = ((1u << 27) - 1u) & ~(1u << 13);

// Descriptor handed to the kernels by value.
struct Frac3Dev {
  uint32_t s, k, r;
  uint32_t n;                  // s^r <= 2^30
  uint32_t Wx;                 // compact extents; W_y * W_z < 2^32
  uint32_t Wy, Wz;
  uint64_t cells;              // k^r <= 2^40
  uint64_t plane;              // W_x * W_y
  FastDiv divk, divs, divWx, divWy;
  uint32_t nbhd;               // bit (dz+1)*9 + (dy+1)*3 + (dx+1) selects offset (dx, dy, dz)
  uint32_t birth, survive;     // 27-bit masks over the alive-neighbour count
  uint8_t tau[3][256];         // H_lambda per axis: tau(beta) = (tau[0][b], tau[1][b], tau[2][b])
  uint8_t hnu[512];            // H_nu[(t_z * s + t_y) * s + t_x] = beta, or kHole
};

// Tables staged in shared memory.
struct Tables3 {
  uint8_t tau[3][256];
  uint8_t hnu[512];
};

// Compact coordinates of omega < cells.
__host__ __device__ inline void split3(const Frac3Dev &f, uint64_t omega, uint32_t &wx,
                                       uint32_t &wy, uint32_t &wz) {
  const uint32_t row = (omega >> 32) ? (uint32_t)(omega / f.Wx) : fdiv(f.divWx, (uint32_t)omega);
  wx = (uint32_t)(omega - (uint64_t)row * f.Wx);
  wz = fdiv(f.divWy, row);
  wy = row - wz * f.Wy;
}

// One level of lambda: the low base-k digit of `w` is the replica id, whose
// offset, scaled by s^(mu-1), adds to the point.
__host__ __device__ inline void lambda_level(const Frac3Dev &f, const Tables3 &t, uint32_t &w,
                                             uint32_t scale, uint32_t &X, uint32_t &Y,
                                             uint32_t &Z) {
  const uint32_t q = fdiv(f.divk, w), beta = w - q * f.k;
  w = q;
  X += t.tau[0][beta] * scale;
  Y += t.tau[1][beta] * scale;
  Z += t.tau[2][beta] * scale;
}

// lambda: levels 1, 2, 3, 4, ... take their replica ids from w_x, w_y, w_z,
// w_x, ... in turn.
__host__ __device__ inline void lambda3(const Frac3Dev &f, const Tables3 &t, uint32_t wx,
                                        uint32_t wy, uint32_t wz, uint32_t &x, uint32_t &y,
                                        uint32_t &z) {
  uint32_t X = 0, Y = 0, Z = 0, scale = 1;
  for (uint32_t mu = 1; mu <= f.r; mu += 3) {
    lambda_level(f, t, wx, scale, X, Y, Z);
    scale *= f.s;
    if (mu + 1 > f.r) break;
    lambda_level(f, t, wy, scale, X, Y, Z);
    scale *= f.s;
    if (mu + 2 > f.r) break;
    lambda_level(f, t, wz, scale, X, Y, Z);
    scale *= f.s;
  }
  x = X;
  y = Y;
  z = Z;
}

// nu: per level the base-s digit triple selects a replica id through H_nu (a
// hole rejects the point), which goes into the next base-k digit of its axis.
__host__ __device__ inline bool nu3(const Frac3Dev &f, const Tables3 &t, int32_t x, int32_t y,
                                    int32_t z, uint64_t &omega) {
  if (x < 0 || y < 0 || z < 0 || (uint32_t)x >= f.n || (uint32_t)y >= f.n || (uint32_t)z >= f.n)
    return false;
  uint32_t ux = (uint32_t)x, uy = (uint32_t)y, uz = (uint32_t)z;
  uint32_t w[3] = {0, 0, 0};
  uint32_t wt[3] = {1, 1, 1};
  uint32_t axis = 0;
  for (uint32_t mu = 1; mu <= f.r; ++mu) {
    const uint32_t qx = fdiv(f.divs, ux), qy = fdiv(f.divs, uy), qz = fdiv(f.divs, uz);
    const uint32_t tx = ux - qx * f.s, ty = uy - qy * f.s, tz = uz - qz * f.s;
    ux = qx;
    uy = qy;
    uz = qz;
    const uint32_t id = t.hnu[(tz * f.s + ty) * f.s + tx];
    if (id == kHole) return false;
    if (axis == 0) {
      w[0] += id * wt[0];
      wt[0] *= f.k;
    } else if (axis == 1) {
      w[1] += id * wt[1];
      wt[1] *= f.k;
    } else {
      w[2] += id * wt[2];
      wt[2] *= f.k;
    }
    axis = axis == 2 ? 0 : axis + 1;
  }
  omega = ((uint64_t)w[2] * f.Wy + w[1]) * f.Wx + w[0];
  return true;
}

// A cell's level-1 digits, shared by all of its neighbour walks.
struct Cell3 {
  uint32_t rx, wy, wz;     // w_x without its lowest base-k digit; w_y; w_z
  uint32_t b1;             // level-1 replica id (lowest base-k digit of w_x)
  int t1x, t1y, t1z;       // tau(b1)
};

__host__ __device__ inline Cell3 cell3(const Frac3Dev &f, const Tables3 &t, uint32_t wx,
                                       uint32_t wy, uint32_t wz) {
  Cell3 c;
  c.rx = fdiv(f.divk, wx);
  c.b1 = wx - c.rx * f.k;
  c.wy = wy;
  c.wz = wz;
  c.t1x = t.tau[0][c.b1];
  c.t1y = t.tau[1][c.b1];
  c.t1z = t.tau[2][c.b1];
  return c;
}

// Move one digit by a carry in {-1, 0, 1}: returns the new digit in [0, s)
// and leaves the outgoing carry in `carry`.
__host__ __device__ inline int carry_digit(int digit, int &carry, int s) {
  int v = digit + carry;
  carry = v < 0 ? -1 : (v >= s ? 1 : 0);
  return v - carry * s;
}

// One level of the neighbour walk: the replica id is the low base-k digit
// of `rem` (the compact coordinate this level cycles to), its offset moves by
// the carries, H_nu gives the new id and that level's term of omega (weight
// `wg`) is corrected.  Returns 0 for a hole, 1 when no carry is left, 2 to go
// on to the next level.
__host__ __device__ inline int walk_level(const Frac3Dev &f, const Tables3 &t, uint32_t &rem,
                                          uint64_t &wg, int &cx, int &cy, int &cz,
                                          int64_t &delta) {
  const int s = (int)f.s;
  const uint32_t q = fdiv(f.divk, rem), beta = rem - q * f.k;
  rem = q;
  const int xd = carry_digit(t.tau[0][beta], cx, s), yd = carry_digit(t.tau[1][beta], cy, s),
            zd = carry_digit(t.tau[2][beta], cz, s);
  const uint32_t id = t.hnu[(zd * s + yd) * s + xd];
  if (id == kHole) return 0;
  delta += ((int64_t)id - (int64_t)beta) * (int64_t)wg;
  wg *= f.k;
  return (cx | cy | cz) == 0 ? 1 : 2;
}

// Change of the compact index from the cell to the point (dx, dy, dz) away
// (|d| <= 1), or false for a hole or a point off the box.  nu of the moved
// point differs from the cell's digits only up to the level where the carries
// of all three coordinates stop, so the walk (the digit form of nu) runs from
// level 1 only that far.
__host__ __device__ inline bool neighbour3(const Frac3Dev &f, const Tables3 &t, const Cell3 &c,
                                           int dx, int dy, int dz, int64_t &delta) {
  const int s = (int)f.s;
  int cx = dx, cy = dy, cz = dz;
  const int xd = carry_digit(c.t1x, cx, s), yd = carry_digit(c.t1y, cy, s),
            zd = carry_digit(c.t1z, cz, s);
  const uint32_t id = t.hnu[(zd * s + yd) * s + xd];
  if (id == kHole) return false;
  delta = (int64_t)id - (int64_t)c.b1;
  if ((cx | cy | cz) == 0) return true;
  // levels 2, 3, 4, ... cycle over w_y, w_z, w_x (w_x without its lowest digit)
  uint32_t rx = c.rx, ry = c.wy, rz = c.wz;
  uint64_t wgx = f.k, wgy = f.Wx, wgz = f.plane;
  for (uint32_t mu = 2; mu <= f.r; mu += 3) {
    int st = walk_level(f, t, ry, wgy, cx, cy, cz, delta);
    if (st != 2) return st == 1;
    if (mu + 1 > f.r) break;
    st = walk_level(f, t, rz, wgz, cx, cy, cz, delta);
    if (st != 2) return st == 1;
    if (mu + 2 > f.r) break;
    st = walk_level(f, t, rx, wgx, cx, cy, cz, delta);
    if (st != 2) return st == 1;
  }
  return false;   // a carry out of the top level leaves the box
}

}  // namespace sq3

// ---- the bit-sliced tile kernel (tile3d.cu), host side ----------------------
struct Tile3Program;
// Tile shape of level L (rows of 8 or 16 cells, W_x a multiple of 16, at most
// 4096 slot words), or false when the tile kernel cannot take this level.
bool sq3_tile_shape(const sq3::Frac3Dev &f, uint32_t L, uint32_t &TX, uint32_t &TY,
                    uint32_t &TZ, uint32_t &slots, uint64_t &box);
// The largest level whose program has at most 1024 slot words, or 0 if none.
uint32_t sq3_tile_default_level(const sq3::Frac3Dev &f);
int sq3_tile_prepare(const sq3::Frac3Dev &f, uint32_t L, int device, Tile3Program **out);
void sq3_tile_free(Tile3Program *p);
int sq3_tile_launch(const Tile3Program *p, uint32_t birth, uint32_t survive, int *status,
                    const uint8_t *in, uint8_t *out, cudaStream_t st);
