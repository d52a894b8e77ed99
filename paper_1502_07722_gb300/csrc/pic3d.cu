// The PIC cycle with the pair-potential force in three dimensions (3D3V): the same method as the
// 2D kernels with Eqs. (1)-(3) along x, y and z (the cubic lattice's six neighbours), trilinear
// weights, Esirkepov's 3D current and the 3D Yee scheme. x and y are periodic, z has walls.
// Fixed point: 2^14 per axis (a particle's weight product is at most 2^42). Grids are
// (nz+1) x ny x nx, index (k*ny + j)*nx + i. Yee positions: Ex (i+1/2,j,k), Ey (i,j+1/2,k),
// Ez (i,j,k+1/2), Bx (i,j+1/2,k+1/2), By (i+1/2,j,k+1/2), Bz (i+1/2,j+1/2,k).
//
// The particle kernel stages each tile's fields and node density in shared memory and streams the
// tile's particles straight from their records in coalesced order (the next record's position is
// loaded one iteration ahead); the cell sort stores each block of 256 of a tile's cell-ordered
// particles column by column as a 32-row matrix, so the lanes of a warp hold particles 8 places
// apart in the cell order (neighbouring cells). CTAs draw tiles from a ticket counter (dynamic
// assignment: 10.46 -> 8.79 ms per launch on the 384^2 x 256 slab against a static round robin).
// Deposits use global 64-bit reductions, which are native in L2.
#include <atomic>

#include "pic_device.cuh"

namespace gbpic {

// The kernel instances: Eq. (3), the altered potential and the Morse form, on the cubic and the
// HCP lattice, and the embedded-atom form on the cubic lattice (potential code in bits 0-1,
// kLatHcp in bit 2).
#define GBPIC_FOR_EACH_POT3(X) X(kPotLJ) X(kPotAlt) X(kPotMorse) X(kPotEam) X(kPotLJ | kLatHcp) \
    X(kPotAlt | kLatHcp) X(kPotMorse | kLatHcp)

constexpr int kQ3Bits = 14;
constexpr int kQ3 = 1 << kQ3Bits;
constexpr int kBlock3 = 256;

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ int qoff3(float f) { return __float2int_rn(f * 16384.0f); }

__device__ __forceinline__ void hat3q(int d, int& s0, int& s1, int& s2)
{
    s0 = max(0, kQ3 - d);
    s1 = kQ3 - abs(d - kQ3);
    s2 = max(0, d - kQ3);
}

struct Geo3 {
    int nx, ny, nz;
    unsigned mag_x, mag_y;     // floor(2^32 / nx), floor(2^32 / ny)
};

__device__ __forceinline__ void split3(int cell, const Geo3& g, int& i, int& j, int& k)
{
    unsigned q = __umulhi((unsigned)cell, g.mag_x);
    int r = cell - (int)q * g.nx;
    if (r >= g.nx) { q++; r -= g.nx; }
    i = r;
    unsigned q2 = __umulhi(q, g.mag_y);
    int r2 = (int)q - (int)q2 * g.ny;
    if (r2 >= g.ny) { q2++; r2 -= g.ny; }
    j = r2;
    k = (int)q2;
}

__device__ __forceinline__ size_t idx3(const Geo3& g, int i, int j, int k)
{
    return ((size_t)k * g.ny + j) * g.nx + i;
}

// staggered trilinear gather; (hx, hy, hz) = 1 where the component sits half a cell up
__device__ __forceinline__ float gather3(const float* __restrict__ A, const Geo3& g, int i, int j, int k, float fx,
                                         float fy, float fz, int hx, int hy, int hz)
{
    int i0 = i, j0 = j, r0 = k, r1 = k + 1;
    float wx = fx, wy = fy, wz = fz;
    if (hx) {
        if (fx >= 0.5f) wx = fx - 0.5f;
        else { i0 = wrapn(i - 1, g.nx); wx = fx + 0.5f; }
    }
    if (hy) {
        if (fy >= 0.5f) wy = fy - 0.5f;
        else { j0 = wrapn(j - 1, g.ny); wy = fy + 0.5f; }
    }
    if (hz) {
        if (fz >= 0.5f) {
            wz = fz - 0.5f;
            if (k >= g.nz - 1) { r0 = g.nz - 2; r1 = g.nz - 1; wz = 1.0f; }
        } else if (k >= 1) {
            r0 = k - 1; r1 = k; wz = fz + 0.5f;
        } else {
            r0 = 0; r1 = 1; wz = 0.0f;
        }
    }
    const int i1 = wrapn(i0 + 1, g.nx), j1 = wrapn(j0 + 1, g.ny);
    const float a000 = __ldg(A + idx3(g, i0, j0, r0)), a100 = __ldg(A + idx3(g, i1, j0, r0));
    const float a010 = __ldg(A + idx3(g, i0, j1, r0)), a110 = __ldg(A + idx3(g, i1, j1, r0));
    const float a001 = __ldg(A + idx3(g, i0, j0, r1)), a101 = __ldg(A + idx3(g, i1, j0, r1));
    const float a011 = __ldg(A + idx3(g, i0, j1, r1)), a111 = __ldg(A + idx3(g, i1, j1, r1));
    const float b00 = a000 + wx * (a100 - a000), b10 = a010 + wx * (a110 - a010);
    const float b01 = a001 + wx * (a101 - a001), b11 = a011 + wx * (a111 - a011);
    const float c0 = b00 + wy * (b10 - b00), c1 = b01 + wy * (b11 - b01);
    return c0 + wz * (c1 - c0);
}

// trilinear node density (units n0) and its exact gradient (units n0 per cell); wall rows doubled
__device__ __forceinline__ void density3(const u64* __restrict__ rho, const Geo3& g, float rho_s, int i, int j, int k,
                                         float fx, float fy, float fz, float& n, float* grad)
{
    const int i1 = wrapn(i + 1, g.nx), j1 = wrapn(j + 1, g.ny);
    float v[8];
#pragma unroll
    for (int c = 0; c < 2; c++)
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int a = 0; a < 2; a++) {
                long long r = (long long)__ldg(rho + idx3(g, a ? i1 : i, b ? j1 : j, k + c));
                if (k + c == 0 || k + c == g.nz) r *= 2;
                v[c * 4 + b * 2 + a] = rho_s * (float)r;
            }
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    // along x: differences of the x-pairs weighted in y and z
    const float dx00 = v[1] - v[0], dx10 = v[3] - v[2], dx01 = v[5] - v[4], dx11 = v[7] - v[6];
    grad[0] = gz * (gy * dx00 + fy * dx10) + fz * (gy * dx01 + fy * dx11);
    const float dy00 = v[2] - v[0], dy10 = v[3] - v[1], dy01 = v[6] - v[4], dy11 = v[7] - v[5];
    grad[1] = gz * (gx * dy00 + fx * dy10) + fz * (gx * dy01 + fx * dy11);
    const float dz00 = v[4] - v[0], dz10 = v[5] - v[1], dz01 = v[6] - v[2], dz11 = v[7] - v[3];
    grad[2] = gy * (gx * dz00 + fx * dz10) + fy * (gx * dz01 + fx * dz11);
    n = gz * (gy * (gx * v[0] + fx * v[1]) + fy * (gx * v[2] + fx * v[3])) +
        fz * (gy * (gx * v[4] + fx * v[5]) + fy * (gx * v[6] + fx * v[7]));
}

struct Species3 {
    int32_t* cell;
    float *fx, *fy, *fz, *ux, *uy, *uz;
    const int32_t* tile_start;
    float e_kick, b_rot, p_kick;
    int jsign, pair;
};

struct Args3 {
    Geo3 g;
    int ntiles, nsp, full, pot_mode;
    int T, ntx, nty, W;     // tile edge, tiles along x and y, staged window edge (0: no window)
    float cdt_dx, rho_s, h_coef, c_att, s_rep;
    EamP eam;
    const float* F[6];
    const u64* rho_cur;
    u64* rho_next;
    u64* J[3];
    unsigned* status;
    Species3 sp[2];
};


__device__ __forceinline__ void red64(u64* p, long long v)
{
    if (v != 0) atomicAdd(p, (u64)v);
}

// General 3 x 3 x 3 Esirkepov stencil and node-density change with global reductions.
// (X, Y, Z) global fixed-point coordinates; X1, Y1 may lie outside the periodic range.
__device__ __noinline__ void deposit3_general(Geo3 g, u64* J0, u64* J1, u64* J2, u64* rho_next, int X0, int Y0,
                                              int Z0, int X1, int Y1, int Z1, int jsign, int pair)
{
    const int bx = min(X0, X1) >> kQ3Bits, by = min(Y0, Y1) >> kQ3Bits, bz = min(Z0, Z1) >> kQ3Bits;
    int S0x[3], S1x[3], S0y[3], S1y[3], S0z[3], S1z[3];
    hat3q(X0 - bx * kQ3, S0x[0], S0x[1], S0x[2]);
    hat3q(X1 - bx * kQ3, S1x[0], S1x[1], S1x[2]);
    hat3q(Y0 - by * kQ3, S0y[0], S0y[1], S0y[2]);
    hat3q(Y1 - by * kQ3, S1y[0], S1y[1], S1y[2]);
    hat3q(Z0 - bz * kQ3, S0z[0], S0z[1], S0z[2]);
    hat3q(Z1 - bz * kQ3, S1z[0], S1z[1], S1z[2]);
    // edge sums and weight products in 32-bit (at most 6 * 2^28), widened once per term
    const int sg = jsign;
    for (int c = 0; c < 3; c++)
        for (int b = 0; b < 3; b++) {
            const int jj = wrapn(by + b, g.ny);
            if (jsign) {
                const int P = 2 * S0y[b] * S0z[c] + S1y[b] * S0z[c] + S0y[b] * S1z[c] + 2 * S1y[b] * S1z[c];
                long long acc = 0;
                for (int q = 0; q < 2; q++) {
                    acc -= (long long)(sg * (S1x[q] - S0x[q])) * P;
                    red64(J0 + idx3(g, wrapn(bx + q, g.nx), jj, bz + c), acc);
                }
            }
            if (pair)
                for (int q = 0; q < 3; q++)
                    red64(rho_next + idx3(g, wrapn(bx + q, g.nx), jj, bz + c),
                          (long long)(S1x[q] * S1y[b]) * S1z[c] - (long long)(S0x[q] * S0y[b]) * S0z[c]);
        }
    if (!jsign) return;
    for (int c = 0; c < 3; c++)
        for (int q = 0; q < 3; q++) {
            const int P = 2 * S0x[q] * S0z[c] + S1x[q] * S0z[c] + S0x[q] * S1z[c] + 2 * S1x[q] * S1z[c];
            long long acc = 0;
            for (int b = 0; b < 2; b++) {
                acc -= (long long)(sg * (S1y[b] - S0y[b])) * P;
                red64(J1 + idx3(g, wrapn(bx + q, g.nx), wrapn(by + b, g.ny), bz + c), acc);
            }
        }
    for (int b = 0; b < 3; b++)
        for (int q = 0; q < 3; q++) {
            const int P = 2 * S0x[q] * S0y[b] + S1x[q] * S0y[b] + S0x[q] * S1y[b] + 2 * S1x[q] * S1y[b];
            long long acc = 0;
            for (int c = 0; c < 2; c++) {
                acc -= (long long)(sg * (S1z[c] - S0z[c])) * P;
                red64(J2 + idx3(g, wrapn(bx + q, g.nx), wrapn(by + b, g.ny), bz + c), acc);
            }
        }
}

// A tile's staged window: the six field components and the pair density (units n0, wall rows
// doubled) on W^3 nodes from (ox, oy, oz); x and y wrap, z rows outside 0..nz repeat the edge row
// (the same values the global gathers clamp to).
struct Win3 {
    const float* f;         // component q (Ex, Ey, Ez, Bx, By, Bz) at f + q W^3, density at f + 6 W^3
    int ox, oy, oz, W, WWW;
};

// Window gathers. Every component of a particle reads the corners of one cell of the window: the
// node cell (lx, ly, lz) for an integer-node axis, or that cell shifted one node down along a
// half-node axis when the particle sits in the lower half of its cell (offset o = 0 or -stride,
// weight f -+ 1/2). One base index serves all seven components; with the window edge WC known
// at compile time the corner and component offsets are immediates.
constexpr int kWin3 = 13;               // window edge of the 10-cell tile (compiled-in instances)

struct Axis3 {
    float g, w;       // weights of the lower and upper node (1 - w, w)
};

// trilinear interpolation of the corners of the cell at p (strides sy = W, sz = W^2) on z-pairs of
// corners: each packed FP32x2 operation interpolates the lower and the upper face at once
// (measured on the 384^2 x 256 slab with the deposit below inlined: 7.73 -> 7.44 ms per launch)
__device__ __forceinline__ float trilerp3(const float* p, int sy, int sz, Axis3 x, Axis3 y, Axis3 z)
{
    const float2 gx2 = make_float2(x.g, x.g), wx2 = make_float2(x.w, x.w);
    const float2 Q0 = __ffma2_rn(wx2, make_float2(p[1], p[sz + 1]), __fmul2_rn(gx2, make_float2(p[0], p[sz])));
    const float2 Q1 = __ffma2_rn(wx2, make_float2(p[sy + 1], p[sz + sy + 1]),
                                 __fmul2_rn(gx2, make_float2(p[sy], p[sz + sy])));
    const float2 R = __ffma2_rn(make_float2(y.w, y.w), Q1, __fmul2_rn(make_float2(y.g, y.g), Q0));
    return z.g * R.x + z.w * R.y;
}

// E and B at the particle from the window (out: Ex, Ey, Ez, Bx, By, Bz); base = index of the
// particle's cell in the window
template <int WC>
__device__ __forceinline__ void wfields3(const float* f, int Wr, int base, float fx, float fy, float fz, float* out)
{
    const int W = WC ? WC : Wr, WW = W * W, WWW = WW * W;
    const bool ux = fx >= 0.5f, uy = fy >= 0.5f, uz = fz >= 0.5f;
    const int ox = ux ? 0 : -1, oy = uy ? 0 : -W, oz = uz ? 0 : -WW;
    const Axis3 X{1.0f - fx, fx}, Y{1.0f - fy, fy}, Z{1.0f - fz, fz};
    const float hx = ux ? fx - 0.5f : fx + 0.5f, hy = uy ? fy - 0.5f : fy + 0.5f, hz = uz ? fz - 0.5f : fz + 0.5f;
    const Axis3 HX{1.0f - hx, hx}, HY{1.0f - hy, hy}, HZ{1.0f - hz, hz};
    out[0] = trilerp3(f + base + ox, W, WW, HX, Y, Z);                       // Ex (i+1/2, j, k)
    out[1] = trilerp3(f + WWW + base + oy, W, WW, X, HY, Z);                 // Ey (i, j+1/2, k)
    out[2] = trilerp3(f + 2 * WWW + base + oz, W, WW, X, Y, HZ);             // Ez (i, j, k+1/2)
    out[3] = trilerp3(f + 3 * WWW + base + oy + oz, W, WW, X, HY, HZ);       // Bx (i, j+1/2, k+1/2)
    out[4] = trilerp3(f + 4 * WWW + base + ox + oz, W, WW, HX, Y, HZ);       // By (i+1/2, j, k+1/2)
    out[5] = trilerp3(f + 5 * WWW + base + ox + oy, W, WW, HX, HY, Z);       // Bz (i+1/2, j+1/2, k)
}

// trilinear density and exact gradient from the window (the arithmetic of density3)
template <int WC>
__device__ __forceinline__ void wdensity3(const float* nh, int Wr, int base, float fx, float fy, float fz, float& n,
                                          float* grad)
{
    const int W = WC ? WC : Wr, sy = W, sz = W * W;
    const float* p = nh + base;
    const float v0 = p[0], v1 = p[1], v2 = p[sy], v3 = p[sy + 1];
    const float v4 = p[sz], v5 = p[sz + 1], v6 = p[sz + sy], v7 = p[sz + sy + 1];
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float dz00 = v4 - v0, dz10 = v5 - v1, dz01 = v6 - v2, dz11 = v7 - v3;
    grad[2] = gy * (gx * dz00 + fx * dz10) + fy * (gx * dz01 + fx * dz11);
    // z-pairs (v0, v4), (v1, v5), (v2, v6), (v3, v7); a difference b - a is fma(-1, a, b), exact
    const float2 P0 = make_float2(v0, v4), P1 = make_float2(v1, v5), P2 = make_float2(v2, v6),
                 P3 = make_float2(v3, v7), m1 = make_float2(-1.0f, -1.0f);
    const float2 gx2 = make_float2(gx, gx), fx2 = make_float2(fx, fx), gy2 = make_float2(gy, gy),
                 fy2 = make_float2(fy, fy);
    const float2 Gx = __ffma2_rn(fy2, __ffma2_rn(m1, P2, P3), __fmul2_rn(gy2, __ffma2_rn(m1, P0, P1)));
    grad[0] = gz * Gx.x + fz * Gx.y;
    const float2 Gy = __ffma2_rn(fx2, __ffma2_rn(m1, P1, P3), __fmul2_rn(gx2, __ffma2_rn(m1, P0, P2)));
    grad[1] = gz * Gy.x + fz * Gy.y;
    const float2 R = __ffma2_rn(fy2, __ffma2_rn(fx2, P3, __fmul2_rn(gx2, P2)),
                                __fmul2_rn(gy2, __ffma2_rn(fx2, P1, __fmul2_rn(gx2, P0))));
    n = gz * R.x + fz * R.y;
}

// rare path (a particle outside its tile's window): everything from global memory.
// out: E x3, B x3, n, grad x3
__device__ __noinline__ void gather_global3(const float* F0, const float* F1, const float* F2, const float* F3,
                                            const float* F4, const float* F5, const u64* rho, Geo3 g, float rho_s,
                                            int fields, int pair, int i, int j, int k, float fx, float fy, float fz,
                                            float* out)
{
    if (fields) {
        out[0] = gather3(F0, g, i, j, k, fx, fy, fz, 1, 0, 0);
        out[1] = gather3(F1, g, i, j, k, fx, fy, fz, 0, 1, 0);
        out[2] = gather3(F2, g, i, j, k, fx, fy, fz, 0, 0, 1);
        out[3] = gather3(F3, g, i, j, k, fx, fy, fz, 0, 1, 1);
        out[4] = gather3(F4, g, i, j, k, fx, fy, fz, 1, 0, 1);
        out[5] = gather3(F5, g, i, j, k, fx, fy, fz, 1, 1, 0);
    }
    if (pair) density3(rho, g, rho_s, i, j, k, fx, fy, fz, out[6], out + 7);
}

// In-cell deposit (the particle stayed in its cell): current on the cell's edges and the node
// density change on its corners, as global 64-bit reductions. Not inlined: it keeps the particle
// loop small enough for the instruction cache.
// A particle that stays in its cell: currents on the cell's edges, node density on its corners.
// The edge sums 2 S0 S0' + S1 S0' + S0 S1' + 2 S1 S1' are formed as S0 (2 S0' + S1') + S1 (S0' + 2 S1')
// from the second axis' two combinations (each product at most 3 * 2^28, the sum at most
// 6 * 2^28 < 2^31: exact in 32-bit); one widening multiply per term. Every reduction is issued
// without a zero test: a particle that moved along an axis almost never has a zero term, and a zero
// adds nothing. Inlined: the currents' base pointers stay kernel parameters (against an
// out-of-line call: 7.68 -> 7.44 ms per launch on the 384^2 x 256 slab).
__device__ __forceinline__ void deposit3_cell(Geo3 g, u64* J0, u64* J1, u64* J2, u64* rho_next, int i, int j,
                                                   int k, int x0, int y0, int z0, int x1, int y1, int z1, int jsign,
                                                   int pair)
{
    const int i1 = wrapn(i + 1, g.nx), j1 = wrapn(j + 1, g.ny);
    // one base index and the offsets to the cell's other corners (x, y periodic)
    const size_t base = idx3(g, i, j, k);
    const ptrdiff_t ox = i1 - i, oy = (ptrdiff_t)(j1 - j) * g.nx, oz = (ptrdiff_t)g.nx * g.ny;
    const int ax0 = kQ3 - x0, ax1 = kQ3 - x1, ay0 = kQ3 - y0, ay1 = kQ3 - y1, az0 = kQ3 - z0, az1 = kQ3 - z1;
    if (jsign) {
        const int dX = jsign * (x1 - x0), dY = jsign * (y1 - y0), dZ = jsign * (z1 - z0);
        // (2 S0' + S1', S0' + 2 S1') of the lower (L) and upper (H) node of y and z
        const int Ly0 = 2 * ay0 + ay1, Ly1 = ay0 + 2 * ay1, Hy0 = 2 * y0 + y1, Hy1 = y0 + 2 * y1;
        const int Lz0 = 2 * az0 + az1, Lz1 = az0 + 2 * az1, Hz0 = 2 * z0 + z1, Hz1 = z0 + 2 * z1;
        if (dX) {
            // J6x(i+1/2, j+b, k+c) = dX (2 S0y S0z + S1y S0z + S0y S1z + 2 S1y S1z)
            atomicAdd(J0 + base, (u64)((long long)dX * (ay0 * Lz0 + ay1 * Lz1)));
            atomicAdd(J0 + base + oy, (u64)((long long)dX * (y0 * Lz0 + y1 * Lz1)));
            atomicAdd(J0 + base + oz, (u64)((long long)dX * (ay0 * Hz0 + ay1 * Hz1)));
            atomicAdd(J0 + base + oy + oz, (u64)((long long)dX * (y0 * Hz0 + y1 * Hz1)));
        }
        if (dY) {
            atomicAdd(J1 + base, (u64)((long long)dY * (ax0 * Lz0 + ax1 * Lz1)));
            atomicAdd(J1 + base + ox, (u64)((long long)dY * (x0 * Lz0 + x1 * Lz1)));
            atomicAdd(J1 + base + oz, (u64)((long long)dY * (ax0 * Hz0 + ax1 * Hz1)));
            atomicAdd(J1 + base + ox + oz, (u64)((long long)dY * (x0 * Hz0 + x1 * Hz1)));
        }
        if (dZ) {
            atomicAdd(J2 + base, (u64)((long long)dZ * (ax0 * Ly0 + ax1 * Ly1)));
            atomicAdd(J2 + base + ox, (u64)((long long)dZ * (x0 * Ly0 + x1 * Ly1)));
            atomicAdd(J2 + base + oy, (u64)((long long)dZ * (ax0 * Hy0 + ax1 * Hy1)));
            atomicAdd(J2 + base + ox + oy, (u64)((long long)dZ * (x0 * Hy0 + x1 * Hy1)));
        }
    }
    if (pair) {
        // the density changes by S(new) - S(old) on each corner; x-y products exact in 32-bit
        const int sx0[2] = {ax0, x0}, sx1[2] = {ax1, x1};
        const int sy0[2] = {ay0, y0}, sy1[2] = {ay1, y1};
        const int sz0[2] = {az0, z0}, sz1[2] = {az1, z1};
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int b = 0; b < 2; b++)
#pragma unroll
                for (int q = 0; q < 2; q++)
                    atomicAdd(rho_next + base + (q ? ox : 0) + (b ? oy : 0) + (c ? oz : 0),
                              (u64)((long long)(sx1[q] * sy1[b]) * sz1[c] - (long long)(sx0[q] * sy0[b]) * sz0[c]));
    }
}

// Particle p of species S (position (cell, fx, fy, fz) loaded by the caller): its momenta are read,
// the record advanced one step and written back before its deposits, so that little state is live
// during them. PAIR is a run-time flag (the pair species): one instance of this code serves both
// species, which keeps the kernel inside the instruction cache. WC is the window edge when it is
// compiled in (0: the run-time a.W).
template <bool FULL, int POT, int WC>
__device__ __forceinline__ void process3(const Args3& a, const Species3& S, const Win3& w, const bool PAIR, int p,
                                         const int cell, const float fx, const float fy, const float fz)
{
    const Geo3& g = a.g;
    float ux = S.ux[p], uy = S.uy[p], uz = S.uz[p];
    int i, j, k;
    split3(cell, g, i, j, k);
    // window coordinates (x, y periodic: the image closest to the window centre)
    const int W = WC ? WC : w.W, cen = W / 2;
    int lx = i - w.ox, ly = j - w.oy;
    if (lx - cen > g.nx / 2) lx -= g.nx;
    else if (cen - lx > g.nx / 2) lx += g.nx;
    if (ly - cen > g.ny / 2) ly -= g.ny;
    else if (cen - ly > g.ny / 2) ly += g.ny;
    const int lz = k - w.oz;
    const bool inwin = W > 0 && lx >= 1 && lx + 2 < W && ly >= 1 && ly + 2 < W && lz >= 1 && lz + 2 < W;
    float kx = 0.f, ky = 0.f, kz = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    float n = 0.f, gr[3] = {0.f, 0.f, 0.f};
    if (inwin) {
        const int Wk = WC ? WC : W;
        const int base = (lz * Wk + ly) * Wk + lx;
        if (FULL) {
            float o[6];
            wfields3<WC>(w.f, W, base, fx, fy, fz, o);
            kx = S.e_kick * o[0]; ky = S.e_kick * o[1]; kz = S.e_kick * o[2];
            bx = o[3]; by = o[4]; bz = o[5];
        }
        if (PAIR) wdensity3<WC>(w.f + 6 * (WC ? WC * WC * WC : w.WWW), W, base, fx, fy, fz, n, gr);
    } else {
        float o[10];
        gather_global3(a.F[0], a.F[1], a.F[2], a.F[3], a.F[4], a.F[5], a.rho_cur, g, a.rho_s, FULL ? 1 : 0,
                       PAIR ? 1 : 0, i, j, k, fx, fy, fz, o);
        if (FULL) {
            kx = S.e_kick * o[0]; ky = S.e_kick * o[1]; kz = S.e_kick * o[2];
            bx = o[3]; by = o[4]; bz = o[5];
        }
        if (PAIR) { n = o[6]; gr[0] = o[7]; gr[1] = o[8]; gr[2] = o[9]; }
    }
    if (PAIR) {
        if (n > 0.0f) {
            const float c = fast_cbrt(n);
            const float inv43 = fast_rcp(n * c);
            float pf[3];
            pair_force3<POT>(n, c, inv43, gr, a.h_coef, a.pot_mode, a.c_att, a.s_rep, pf, a.eam);
            kx += S.p_kick * pf[0];
            ky += S.p_kick * pf[1];
            kz += S.p_kick * pf[2];
        }
    }
    const float ux0 = ux, uy0 = uy, uz0 = uz;
    ux += kx; uy += ky; uz += kz;
    if (FULL) {
        const float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        const float tx = S.b_rot * ig * bx, ty = S.b_rot * ig * by, tz = S.b_rot * ig * bz;
        const float s = 2.0f * fast_rcp(1.0f + tx * tx + ty * ty + tz * tz);
        const float px = ux + (uy * tz - uz * ty);
        const float py = uy + (uz * tx - ux * tz);
        const float pz = uz + (ux * ty - uy * tx);
        ux += s * (py * tz - pz * ty);
        uy += s * (pz * tx - px * tz);
        uz += s * (px * ty - py * tx);
    }
    ux += kx; uy += ky; uz += kz;
    const float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
    float dxi = ux * a.cdt_dx * ig, dyi = uy * a.cdt_dx * ig, dze = uz * a.cdt_dx * ig;
    if (!(fabsf(dxi) < 1.0f && fabsf(dyi) < 1.0f && fabsf(dze) < 1.0f)) {
        atomicOr(a.status, (isfinite(ux) && isfinite(uy) && isfinite(uz)) ? kErrMove : kErrNan);
        ux = ux0; uy = uy0; uz = uz0; dxi = dyi = dze = 0.0f;
    }
    float nfx = fx + dxi, nfy = fy + dyi, nfz = fz + dze;
    int di = (int)floorf(nfx);
    nfx -= (float)di;
    if (nfx >= 1.0f) { nfx = 0.0f; di += 1; }
    int dj = (int)floorf(nfy);
    nfy -= (float)dj;
    if (nfy >= 1.0f) { nfy = 0.0f; dj += 1; }
    int dk = 0;
    if (k == 0 && nfz < 0.0f) {
        nfz = -nfz; uz = -uz;
    } else if (k == g.nz - 1 && nfz >= 1.0f) {
        nfz = 2.0f - nfz; uz = -uz;
    } else {
        dk = (int)floorf(nfz);
        nfz -= (float)dk;
        if (nfz >= 1.0f) { nfz = 0.0f; dk += 1; }
    }
    S.cell[p] = (int)idx3(g, wrapn(i + di, g.nx), wrapn(j + dj, g.ny), k + dk);
    S.fx[p] = nfx;
    S.fy[p] = nfy;
    S.fz[p] = nfz;
    S.ux[p] = ux;
    S.uy[p] = uy;
    S.uz[p] = uz;

    const int x0 = qoff3(fx), x1 = qoff3(nfx), y0 = qoff3(fy), y1 = qoff3(nfy), z0 = qoff3(fz), z1 = qoff3(nfz);
    const bool moved = (di | dj | dk) != 0 || x1 != x0 || y1 != y0 || z1 != z0;
    if (!moved) return;
    if ((di | dj | dk) == 0) {
        deposit3_cell(g, a.J[0], a.J[1], a.J[2], a.rho_next, i, j, k, x0, y0, z0, x1, y1, z1, S.jsign, PAIR ? 1 : 0);
    } else {
        deposit3_general(g, a.J[0], a.J[1], a.J[2], a.rho_next, i * kQ3 + x0, j * kQ3 + y0, k * kQ3 + z0,
                         (i + di) * kQ3 + x1, (j + dj) * kQ3 + y1, (k + dk) * kQ3 + z1, S.jsign, PAIR ? 1 : 0);
    }
}

template <bool FULL, int POT, int WC>
__global__ void __launch_bounds__(kBlock3, 3) k_particles3(const __grid_constant__ Args3 a)
{
    extern __shared__ unsigned smem3[];
    const int W = WC ? WC : a.W, WW = W * W, WWW = WW * W;
    Win3 w;
    w.W = W;
    float* wf = reinterpret_cast<float*>(smem3);
    w.f = wf;
    w.WWW = WWW;
    const Geo3& g = a.g;
    // tiles are handed out dynamically from the ticket counter in the status words (atomicInc wraps
    // it back to 0 once every CTA has drawn its last, failing, ticket)
    __shared__ int slot;
    for (;;) {
        if (threadIdx.x == 0) slot = (int)atomicInc(a.status + 2, (unsigned)(a.ntiles + gridDim.x - 1));
        __syncthreads();
        const int t = slot;
        __syncthreads();
        if (t >= a.ntiles) break;
        int cnt = 0;
        for (int s = 0; s < a.nsp; s++) cnt += a.sp[s].tile_start[t + 1] - a.sp[s].tile_start[t];
        if (cnt == 0) continue;
        const int tx = t % a.ntx, ty = (t / a.ntx) % a.nty, tz = t / (a.ntx * a.nty);
        w.ox = tx * a.T - 1;
        w.oy = ty * a.T - 1;
        w.oz = tz * a.T - 1;
        if (W > 0) {
            __syncthreads();                       // the previous tile is done with the window
            for (int q = threadIdx.x; q < WWW; q += blockDim.x) {
                const int c = q / WW, r = q - c * WW, b = r / W, e = r - b * W;
                int gx = (w.ox + e) % g.nx, gy = (w.oy + b) % g.ny;
                gx = gx < 0 ? gx + g.nx : gx;
                gy = gy < 0 ? gy + g.ny : gy;
                const int gz = w.oz + c;
                const int gn = min(max(gz, 0), g.nz), gh = min(max(gz, 0), g.nz - 1);
                const size_t in = idx3(g, gx, gy, gn), ih = idx3(g, gx, gy, gh);
                if (FULL) {
                    wf[q] = __ldg(a.F[0] + in);
                    wf[WWW + q] = __ldg(a.F[1] + in);
                    wf[2 * WWW + q] = __ldg(a.F[2] + ih);
                    wf[3 * WWW + q] = __ldg(a.F[3] + ih);
                    wf[4 * WWW + q] = __ldg(a.F[4] + ih);
                    wf[5 * WWW + q] = __ldg(a.F[5] + in);
                }
                const long long r0 = (long long)__ldg(a.rho_cur + in);
                wf[6 * WWW + q] = a.rho_s * (float)((gn == 0 || gn == g.nz) ? 2 * r0 : r0);
            }
            __syncthreads();
        }
#pragma unroll 1
        for (int s = 0; s < 2; s++) {
            if (s >= a.nsp) break;
            const Species3& S = a.sp[s];
            const int p0 = S.tile_start[t], p1 = S.tile_start[t + 1];
            // consecutive threads take consecutive records (coalesced); the cell sort's block
            // layout gives a warp's lanes neighbouring cells
            // the next record's position is loaded one iteration ahead (its first use is at the top
            // of the iteration); the momenta, first used after the gathers, are loaded in the iteration
            int ncell = 0;
            float nfx = 0.0f, nfy = 0.0f, nfz = 0.0f;
            if (p0 + (int)threadIdx.x < p1) {
                const int q = p0 + (int)threadIdx.x;
                ncell = S.cell[q]; nfx = S.fx[q]; nfy = S.fy[q]; nfz = S.fz[q];
            }
            for (int p = p0 + (int)threadIdx.x; p < p1; p += kBlock3) {
                const int cell = ncell;
                const float fx = nfx, fy = nfy, fz = nfz;
                if (p + kBlock3 < p1) {
                    const int q = p + kBlock3;
                    ncell = S.cell[q]; nfx = S.fx[q]; nfy = S.fy[q]; nfz = S.fz[q];
                }
                process3<FULL, POT, WC>(a, S, w, S.pair != 0, p, cell, fx, fy, fz);
            }
        }
    }
}

static Geo3 geo_of(const Ctx& c)
{
    Geo3 g;
    g.nx = c.nx;
    g.ny = c.ny;
    g.nz = c.nz;
    g.mag_x = (unsigned)(4294967296ULL / (unsigned long long)c.nx);
    g.mag_y = (unsigned)(4294967296ULL / (unsigned long long)c.ny);
    return g;
}

void launch_particle_step3(Ctx& c, cudaStream_t st)
{
    Args3 a;
    memset(&a, 0, sizeof(a));
    a.g = geo_of(c);
    a.ntiles = c.ntiles;
    a.nsp = c.nsp;
    a.full = c.cfg.mode == PIC_MODE_FULL;
    a.pot_mode = pot_code(c.cfg);
    a.cdt_dx = (float)(kC * c.dt / c.cfg.dx);
    a.rho_s = (float)c.rho_scale;
    a.h_coef = (float)(c.r0 / (6.0 * c.cfg.dx));
    a.c_att = pot_param(c.cfg);
    a.s_rep = (float)c.cfg.s_rep;
    a.eam = eam_params(c.cfg);
    for (int q = 0; q < 6; q++) a.F[q] = c.F[q];
    a.rho_cur = c.rho[c.cur];
    a.rho_next = c.rho[1 - c.cur];
    for (int q = 0; q < 3; q++) a.J[q] = c.J[q];
    a.status = c.status;
    for (int s = 0; s < 2; s++) {
        const Species& S = c.sp[s];
        Species3& d = a.sp[s];
        d.cell = S.a.cell; d.fx = S.a.fx; d.fy = S.a.fy; d.fz = S.a.fz;
        d.ux = S.a.ux; d.uy = S.a.uy; d.uz = S.a.uz;
        d.tile_start = S.tile_start;
        d.e_kick = S.e_kick; d.b_rot = S.b_rot; d.p_kick = S.p_kick;
        d.jsign = S.jsign; d.pair = S.pair;
    }
    a.T = c.T;
    a.ntx = c.ntx;
    a.nty = c.nty;
    // window of the tile plus one node below and two above on each axis; staged when three CTAs
    // still fit on one SM
    const int W = c.T + 3;
    a.W = (size_t)7 * W * W * W * 4 <= 72 * 1024 ? W : 0;
    const size_t shmem = sizeof(unsigned) * ((size_t)7 * a.W * a.W * a.W);
    // the attributes are per device: remember what each device has been given
    static std::atomic<size_t> configured[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    if (shmem > configured[dev].load()) {
#define GBPIC_ATTR(P)                                                                                   \
        for (const void* k : {(const void*)k_particles3<true, (P), 0>, (const void*)k_particles3<false, (P), 0>, \
                              (const void*)k_particles3<true, (P), kWin3>,                                   \
                              (const void*)k_particles3<false, (P), kWin3>}) {                               \
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);           \
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);                \
        }
        GBPIC_FOR_EACH_POT3(GBPIC_ATTR)
#undef GBPIC_ATTR
        configured[dev].store(shmem);
    }
    int grid = c.ntiles < c.nsm * 3 ? c.ntiles : c.nsm * 3;
    if (grid < 1) grid = 1;
    // the instance with the potential and the lattice compiled in, and the window edge when it is
    // the 10-cell tile's
    const bool wc = a.W == kWin3;
    switch ((a.pot_mode & 7) | (a.full ? 8 : 0)) {
#define GBPIC_CASE(P)                                                                                         \
    case 8 | (P):                                                                                             \
        if (wc) k_particles3<true, (P), kWin3><<<grid, kBlock3, shmem, st>>>(a);                              \
        else k_particles3<true, (P), 0><<<grid, kBlock3, shmem, st>>>(a);                                     \
        break;                                                                                                \
    case (P):                                                                                                 \
        if (wc) k_particles3<false, (P), kWin3><<<grid, kBlock3, shmem, st>>>(a);                             \
        else k_particles3<false, (P), 0><<<grid, kBlock3, shmem, st>>>(a);                                    \
        break;
        GBPIC_FOR_EACH_POT3(GBPIC_CASE)
#undef GBPIC_CASE
    }
}

// ---- stand-alone node density and pair force ------------------------------------------------

__global__ void k_deposit_density3(const int32_t* __restrict__ cell, const float* __restrict__ fx,
                                   const float* __restrict__ fy, const float* __restrict__ fz, int64_t n, Geo3 g,
                                   u64* out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        split3(cell[p], g, i, j, k);
        const long long x = qoff3(fx[p]), y = qoff3(fy[p]), z = qoff3(fz[p]);
        const long long sx[2] = {kQ3 - x, x}, sy[2] = {kQ3 - y, y}, sz[2] = {kQ3 - z, z};
        const int i1 = wrapn(i + 1, g.nx), j1 = wrapn(j + 1, g.ny);
        for (int c = 0; c < 2; c++)
            for (int b = 0; b < 2; b++)
                for (int q = 0; q < 2; q++) red64(out + idx3(g, q ? i1 : i, b ? j1 : j, k + c), sx[q] * sy[b] * sz[c]);
    }
}

__global__ void k_pair_force3(const int32_t* __restrict__ cell, const float* __restrict__ fx,
                              const float* __restrict__ fy, const float* __restrict__ fz, int64_t n, Geo3 g,
                              const u64* __restrict__ rho, float rho_s, float h_coef, int pot_mode, float c_att,
                              float s_rep, float f_unit, EamP eam, float* __restrict__ out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        split3(cell[p], g, i, j, k);
        float dens, gr[3];
        density3(rho, g, rho_s, i, j, k, fx[p], fy[p], fz[p], dens, gr);
        float F[3] = {0.f, 0.f, 0.f};
        if (dens > 0.0f) {
            const float cr = fast_cbrt(dens);
            const float inv43 = fast_rcp(dens * cr);
            pair_force3(dens, cr, inv43, gr, h_coef, pot_mode, c_att, s_rep, F, eam);
            for (int d = 0; d < 3; d++) F[d] *= f_unit;
        }
        out[3 * p] = F[0];
        out[3 * p + 1] = F[1];
        out[3 * p + 2] = F[2];
    }
}

static int grid3(const Ctx& c, int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)c.nsm * 8) g = (int64_t)c.nsm * 8;
    return g < 1 ? 1 : (int)g;
}

void launch_deposit_density3(Ctx& c, u64* out, cudaStream_t st)
{
    cudaMemsetAsync(out, 0, sizeof(u64) * c.nn, st);
    const Species& S = c.sp[0];
    if (S.n == 0) return;
    k_deposit_density3<<<grid3(c, S.n), 256, 0, st>>>(S.a.cell, S.a.fx, S.a.fy, S.a.fz, S.n, geo_of(c), out);
}

void launch_pair_force3(Ctx& c, float* out, cudaStream_t st)
{
    const Species& S = c.sp[0];
    if (S.n == 0) return;
    k_pair_force3<<<grid3(c, S.n), 256, 0, st>>>(S.a.cell, S.a.fx, S.a.fy, S.a.fz, S.n, geo_of(c), c.rho[c.cur],
                                                  (float)c.rho_scale, (float)(c.r0 / (6.0 * c.cfg.dx)),
                                                  pot_code(c.cfg), pot_param(c.cfg), (float)c.cfg.s_rep,
                                                  (float)(c.D / c.r0), eam_params(c.cfg), out);
}

// ---- 3D Yee --------------------------------------------------------------------------------

struct Field3 {
    Geo3 g;
    int k_ant;
    float h_b, h_e, cj, mur;
    float* F[6];
    const u64* J[3];
    float* save;          // 8 planes of nx*ny: Ex(0) Ex(1) Ex(nz-1) Ex(nz) Ey(0) Ey(1) Ey(nz-1) Ey(nz)
    const float* antc;    // nx*ny
    const float* ants;
    const float* ant;
    int k_flux;           // node plane below the antenna (Poynting flux of the injected energy)
    double* flux;
};

__global__ void k_half_B3(const Field3 f, int save)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const Geo3& g = f.g;
    if (i >= g.nx) return;
    const int ip = i + 1 == g.nx ? 0 : i + 1, jp = j + 1 == g.ny ? 0 : j + 1;
    const size_t c = idx3(g, i, j, k);
    const float *Ex = f.F[0], *Ey = f.F[1], *Ez = f.F[2];
    float *Bx = f.F[3], *By = f.F[4], *Bz = f.F[5];
    const float ex = Ex[c], ey = Ey[c];
    if (k < g.nz) {
        const float ez = Ez[c];
        const size_t up = c + (size_t)g.nx * g.ny;
        Bx[c] += f.h_b * ((Ey[up] - ey) - (Ez[idx3(g, i, jp, k)] - ez));
        By[c] += f.h_b * ((Ez[idx3(g, ip, j, k)] - ez) - (Ex[up] - ex));
    }
    Bz[c] += f.h_b * ((Ex[idx3(g, i, jp, k)] - ex) - (Ey[idx3(g, ip, j, k)] - ey));
    if (save) {
        int slot = -1;
        if (k == 0) slot = 0;
        else if (k == 1) slot = 1;
        else if (k == g.nz - 1) slot = 2;
        else if (k == g.nz) slot = 3;
        if (slot >= 0) {
            const size_t plane = (size_t)g.nx * g.ny, q = (size_t)j * g.nx + i;
            f.save[slot * plane + q] = ex;
            f.save[(4 + slot) * plane + q] = ey;
        }
    }
}

__device__ __forceinline__ float ex3_new(const Field3& f, int i, int j, int k, float old)
{
    const Geo3& g = f.g;
    const size_t c = idx3(g, i, j, k);
    const int jm = j == 0 ? g.ny - 1 : j - 1;
    float v = old + f.h_e * ((f.F[5][c] - f.F[5][idx3(g, i, jm, k)]) - (f.F[4][c] - f.F[4][idx3(g, i, j, k - 1)])) -
              f.cj * (float)(long long)f.J[0][c];
    if (k == f.k_ant) {
        const size_t q = (size_t)j * g.nx + i;
        v += f.antc[q] * f.ant[0] + f.ants[q] * f.ant[1];
    }
    return v;
}
__device__ __forceinline__ float ey3_new(const Field3& f, int i, int j, int k, float old)
{
    const Geo3& g = f.g;
    const size_t c = idx3(g, i, j, k);
    const int im = i == 0 ? g.nx - 1 : i - 1;
    return old + f.h_e * ((f.F[3][c] - f.F[3][idx3(g, i, j, k - 1)]) - (f.F[5][c] - f.F[5][idx3(g, im, j, k)])) -
           f.cj * (float)(long long)f.J[1][c];
}

__global__ void k_E3(const Field3 f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const Geo3& g = f.g;
    float s = 0.0f;            // on the flux plane: this node's (Ex By - Ey Bx) at the half step
    if (i < g.nx) {
        const size_t c = idx3(g, i, j, k), plane = (size_t)g.nx * g.ny, q = (size_t)j * g.nx + i;
        float* Ex = f.F[0];
        float* Ey = f.F[1];
        if (k > 0 && k < g.nz) {
            const float ex0 = Ex[c], ey0 = Ey[c];
            const float ex1 = ex3_new(f, i, j, k, ex0), ey1 = ey3_new(f, i, j, k, ey0);
            Ex[c] = ex1;
            Ey[c] = ey1;
            if (k == f.k_flux)
                s = 0.25f * ((ex0 + ex1) * (f.F[4][c - plane] + f.F[4][c]) -
                             (ey0 + ey1) * (f.F[3][c - plane] + f.F[3][c]));
        } else if (k == 0) {
            const float x0 = f.save[q], x1 = f.save[plane + q], y0 = f.save[4 * plane + q], y1 = f.save[5 * plane + q];
            Ex[c] = x1 + f.mur * (ex3_new(f, i, j, 1, x1) - x0);
            Ey[c] = y1 + f.mur * (ey3_new(f, i, j, 1, y1) - y0);
        } else {
            const float x1 = f.save[2 * plane + q], x0 = f.save[3 * plane + q], y1 = f.save[6 * plane + q],
                        y0 = f.save[7 * plane + q];
            Ex[c] = x1 + f.mur * (ex3_new(f, i, j, g.nz - 1, x1) - x0);
            Ey[c] = y1 + f.mur * (ey3_new(f, i, j, g.nz - 1, y1) - y0);
        }
        if (k < g.nz) {
            const int im = i == 0 ? g.nx - 1 : i - 1, jm = j == 0 ? g.ny - 1 : j - 1;
            f.F[2][c] += f.h_e * ((f.F[4][c] - f.F[4][idx3(g, im, j, k)]) - (f.F[3][c] - f.F[3][idx3(g, i, jm, k)])) -
                         f.cj * (float)(long long)f.J[2][c];
        }
    }
    if (k == f.k_flux) {                                  // uniform over the block
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(f.flux, (double)s);
    }
}

__global__ void k_antenna3(AntennaParams p, long long step, float* ant)
{
    float s = 0.0f, c = 0.0f;
    if (p.on) {
        const double tau = ((double)step + 0.5) * p.dt - p.t_ant;
        const double env = exp(-2.0 * 0.6931471805599453 * tau * tau / (p.tau_fwhm * p.tau_fwhm));
        const double a = p.coef * env;
        s = (float)(a * sin(p.omega * tau));
        c = (float)(a * cos(p.omega * tau));
    }
    ant[0] = s;
    ant[1] = c;
}

void launch_fields3(Ctx& c, cudaStream_t st, int64_t step, int64_t* launches)
{
    Field3 f;
    f.g = geo_of(c);
    f.k_ant = c.k_ant;
    f.h_b = (float)(0.5 * c.dt / c.cfg.dx);
    f.h_e = (float)(kC * kC * c.dt / c.cfg.dx);
    f.cj = (float)(kQe * c.w / (6.0 * 4398046511104.0 * c.cfg.dx * c.cfg.dx * kEps0));
    const double cdt = kC * c.dt;
    f.mur = (float)((cdt - c.cfg.dx) / (cdt + c.cfg.dx));
    for (int q = 0; q < 6; q++) f.F[q] = c.F[q];
    for (int q = 0; q < 3; q++) f.J[q] = c.J[q];
    f.save = c.mur_save;
    f.antc = c.ant_c;
    f.ants = c.ant_s;
    f.ant = c.ant;
    f.k_flux = c.k_ant - 1 >= 1 ? c.k_ant - 1 : -1;
    f.flux = c.red_out + 5;
    k_antenna3<<<1, 1, 0, st>>>(make_antenna_params(c), (long long)step, c.ant);
    dim3 block(256), grid((c.nx + 255) / 256, c.ny, c.nz + 1);
    k_half_B3<<<grid, block, 0, st>>>(f, 1);
    k_E3<<<grid, block, 0, st>>>(f);
    k_half_B3<<<grid, block, 0, st>>>(f, 0);
    if (launches) *launches += 4;
}

// ---- energies ------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_energy3(const Species3 s0, const Species3 s1, int64_t n0, int64_t n1, int nsp, Geo3 g,
                                                 const float* F0, const float* F1, const float* F2, const float* F3,
                                                 const float* F4, const float* F5, const u64* rho, float rho_s,
                                                 float h_coef, int pot_mode, float c_att, float s_rep, EamP eam,
                                                 double* partials)
{
    __shared__ double sh[256];
    const int64_t tid = blockIdx.x * (int64_t)256 + threadIdx.x, stride = (int64_t)gridDim.x * 256;
    double ke[2] = {0.0, 0.0}, pe = 0.0, fe = 0.0, fb = 0.0;
    for (int s = 0; s < nsp; s++) {
        const Species3& S = s == 0 ? s0 : s1;
        const int64_t ns = s == 0 ? n0 : n1;
        for (int64_t p = tid; p < ns; p += stride) {
            const float ux = S.ux[p], uy = S.uy[p], uz = S.uz[p];
            const float u2 = ux * ux + uy * uy + uz * uz;
            ke[s] += (double)(u2 / (sqrtf(1.0f + u2) + 1.0f));
            if (s == 0) {
                int i, j, k;
                split3(S.cell[p], g, i, j, k);
                float dens, gr[3];
                density3(rho, g, rho_s, i, j, k, S.fx[p], S.fy[p], S.fz[p], dens, gr);
                if (dens > 0.0f) {
                    const float cr = fast_cbrt(dens), inv43 = fast_rcp(dens * cr);
                    float e = 0.0f;
                    e += pair_energy3(cr, inv43, gr, h_coef, pot_mode, c_att, s_rep, eam);
                    pe += (double)e;
                }
            }
        }
    }
    const int64_t nn = (int64_t)(g.nz + 1) * g.ny * g.nx, plane = (int64_t)g.ny * g.nx;
    for (int64_t c = tid; c < nn; c += stride) {
        const int k = (int)(c / plane);
        const double wn = (k == 0 || k == g.nz) ? 0.5 : 1.0;
        const double ex = F0[c], ey = F1[c], bz = F5[c];
        fe += wn * (ex * ex + ey * ey);
        fb += wn * bz * bz;
        if (k < g.nz) {
            const double ez = F2[c], bx = F3[c], by = F4[c];
            fe += ez * ez;
            fb += bx * bx + by * by;
        }
    }
    double vals[5] = {ke[0], ke[1], fe, fb, pe};
    for (int q = 0; q < 5; q++) {
        sh[threadIdx.x] = vals[q];
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * 5 + q] = sh[0];
        __syncthreads();
    }
}

__global__ void k_energy3_final(const double* __restrict__ partials, int nb, double* out)
{
    __shared__ double sh[256];
    for (int q = 0; q < 5; q++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += 256) v += partials[(size_t)b * 5 + q];
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sh[0];
        __syncthreads();
    }
}

void launch_energy3(Ctx& c, cudaStream_t st, double* host_out5)
{
    Species3 sp[2];
    memset(sp, 0, sizeof(sp));
    for (int s = 0; s < 2; s++) {
        const Species& S = c.sp[s];
        sp[s].cell = S.a.cell; sp[s].fx = S.a.fx; sp[s].fy = S.a.fy; sp[s].fz = S.a.fz;
        sp[s].ux = S.a.ux; sp[s].uy = S.a.uy; sp[s].uz = S.a.uz;
    }
    const int nb = c.nsm * 4;
    k_energy3<<<nb, 256, 0, st>>>(sp[0], sp[1], c.sp[0].n, c.nsp > 1 ? c.sp[1].n : 0, c.nsp, geo_of(c), c.F[0], c.F[1],
                                  c.F[2], c.F[3], c.F[4], c.F[5], c.rho[c.cur], (float)c.rho_scale,
                                  (float)(c.r0 / (6.0 * c.cfg.dx)), pot_code(c.cfg), pot_param(c.cfg),
                                  (float)c.cfg.s_rep, eam_params(c.cfg), c.partials);
    k_energy3_final<<<1, 256, 0, st>>>(c.partials, nb, c.red_out);
    double raw[5];
    cudaMemcpyAsync(raw, c.red_out, sizeof(raw), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    const double vol = c.cfg.dx * c.cfg.dx * c.cfg.dx, mu0 = 1.0 / (kEps0 * kC * kC);
    host_out5[0] = raw[0] * c.w * c.sp[0].mass * kC * kC;
    host_out5[1] = c.nsp > 1 ? raw[1] * c.w * c.sp[1].mass * kC * kC : 0.0;
    host_out5[2] = 0.5 * kEps0 * raw[2] * vol;
    host_out5[3] = 0.5 / mu0 * raw[3] * vol;
    host_out5[4] = 0.5 * c.D * raw[4] * c.w;
}

}  // namespace gbpic
