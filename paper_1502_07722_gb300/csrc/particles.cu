// The particle kernel of one PIC step (paper, the PIC-cycle paragraph and Fig. 1B):
// for every macroparticle -- gather E, B (Lorentz force) and the node density with its gradient
// (pair-potential force, Eqs. 1-3) -> relativistic Boris push -> move -> charge-conserving
// current deposition (Esirkepov, fixed point) -> node density at the new position.
//
// Work decomposition (GB300):
//  * one CTA owns one tile of T x T cells at a time (particles are sorted into tiles);
//  * the CTA stages a window of (T + 2M + 3)^2 nodes in shared memory: the six field
//    components and the pair density n / n0 in FP32, components of one Yee stagger side by side
//    (one 64-bit load per corner fetches two of them);
//  * thread t of the CTA (128 threads, 8 CTAs per SM) takes the tile's records t, t + 128, ...
//    straight from global memory (coalesced loads and stores, no block barrier); the position of
//    its next record is loaded one iteration ahead. The cell sort
//    stores each block of 1024 of
//    a tile's cell-ordered particles as a 32-row matrix, column by column, so the lanes of a warp
//    hold particles 32 places apart in the cell order: neighbouring cells, whose deposits go to
//    distinct nodes that share cache sectors;
//  * deposits (current, node-density change) are exact 64-bit integer reductions straight into
//    global memory: fire-and-forget on the SM, native in L2. Measured against exact sums in the
//    shared-memory window (32-bit (lo, hi) pairs whose low-word atomic must return the old value
//    for the carry) they are slightly faster and free 17 KB of shared memory per CTA;
//  * the node density is updated incrementally: the next density starts as a copy of the
//    current one and each pair particle adds S(new) - S(old) only when its fixed-point position
//    changed. Ions move ~1e-7 cells per step against a quantum of 1.5e-5 cells, so most of them
//    deposit nothing; the integer result equals a full re-deposit bit for bit;
//  * a particle that stays in its cell (almost all of them) deposits on the four corners of the
//    cell (an electron without per-term zero tests: its terms are almost never zero); a particle
//    that crossed a cell edge uses the 3 x 3 Esirkepov stencil (rare); a particle that drifted
//    beyond the margin since the last sort gathers from global memory (rare);
//  * the code is specialised per species kind (ion, electron, neutral atom) and per potential
//    and lattice, so no per-particle branch tests a species or potential property; Eq. (3) as
//    printed evaluates both in-plane axes at once with packed FP32x2 arithmetic.
// Integer sums make every result independent of the order of the additions.
#include <atomic>

#include "pic_device.cuh"

namespace gbpic {

constexpr int kMargin = 2;              // cells a particle may drift out of its tile between sorts
constexpr int kBlock = 128;                // threads per CTA (8 CTAs per SM)
constexpr int kCtasPerSm = 8;
// The batched kernel reads each slab's arguments from a constant-memory table with a run-time
// index: every use is an indexed constant load into a register, so it needs more registers than
// the single kernel for the same code. At 64 registers it spilled ~100 bytes per thread; at 72
// (7 CTAs per SM) the particle launch of the 16-slab sweep takes 2.03 ms against 2.39 (6 CTAs
// at 80 registers: 2.23).
constexpr int kCtasPerSmBatch = 7;


__device__ __forceinline__ int wrap_any(int i, int nx)
{
    int r = i % nx;
    return r < 0 ? r + nx : r;
}

// The tile's window in shared memory. Field instances keep the components that share a Yee
// stagger side by side, so one 64-bit load fetches both at a corner: (Ex, Bz) at (i + 1/2, k),
// (Ez, Bx) at (i, k + 1/2), (Ey, n / n0) at (i, k), By at (i + 1/2, k + 1/2). Transport
// instances keep n / n0 alone.
struct Window {
    float2* exbz;
    float2* ezbx;
    float2* eyn;
    float* by;
    float* nh;
    int ox, oz, W;
};

// bilinear sum of the corners (c00, c10, c01, c11) of a stagger pair, both components at once
__device__ __forceinline__ float2 bilerp2(float2 c00, float2 c10, float2 c01, float2 c11, float2 gx, float2 wx,
                                          float2 gz, float2 wz)
{
    const float2 b0 = __ffma2_rn(wx, c10, __fmul2_rn(gx, c00));
    const float2 b1 = __ffma2_rn(wx, c11, __fmul2_rn(gx, c01));
    return __ffma2_rn(wz, b1, __fmul2_rn(gz, b0));
}

__device__ __forceinline__ float bilerp1(float c00, float c10, float c01, float c11, float gx, float wx, float gz,
                                         float wz)
{
    const float b0 = __fmaf_rn(wx, c10, __fmul_rn(gx, c00));
    const float b1 = __fmaf_rn(wx, c11, __fmul_rn(gx, c01));
    return __fmaf_rn(wz, b1, __fmul_rn(gz, b0));
}

__device__ __forceinline__ void red64g(u64* p, long long v)
{
    if (v != 0) atomicAdd(p, (u64)v);
}


// exact cell -> (i, k): q = floor(cell / nx) from a multiply-high and one correction
__device__ __forceinline__ void split_cell(int cell, int nx, unsigned magic, int& i, int& k)
{
    unsigned q = __umulhi((unsigned)cell, magic);
    int r = cell - (int)q * nx;
    if (r >= nx) { q++; r -= nx; }
    k = (int)q;
    i = r;
}

// Rare path: fields and node density straight from global memory (particle outside the window).
__device__ __noinline__ void gather_global(const float* F0, const float* F1, const float* F2, const float* F3,
                                           const float* F4, const float* F5, const u64* rho, int nx, int nz,
                                           float rho_s, int full, int pair, int i, int k, float fx, float fz,
                                           float* g)
{
    if (full) {
        g[0] = gather_field(F0, nx, nz, i, k, fx, fz, 1, 0);
        g[1] = gather_field(F1, nx, nz, i, k, fx, fz, 0, 0);
        g[2] = gather_field(F2, nx, nz, i, k, fx, fz, 0, 1);
        g[3] = gather_field(F3, nx, nz, i, k, fx, fz, 0, 1);
        g[4] = gather_field(F4, nx, nz, i, k, fx, fz, 1, 1);
        g[5] = gather_field(F5, nx, nz, i, k, fx, fz, 1, 0);
    }
    if (pair) gather_density(rho, nx, nz, rho_s, i, k, fx, fz, g[6], g[7], g[8]);
}

// Rare path: 3 x 3 Esirkepov stencil and new node density with global atomics. (X, Z) are
// global fixed-point coordinates; X1 may lie outside [0, nx 2^16) (periodic x).
__device__ __noinline__ void deposit_global(u64* rho_next, u64* Jx, u64* Jy, u64* Jz, int nx, int X0, int Z0,
                                            int X1, int Z1, int jsign, int V, int pair)
// pair != 0: the node density changes by S(X1, Z1) - S(X0, Z0)
{
    const int bx = min(X0, X1) >> kQBits, bz = min(Z0, Z1) >> kQBits;
    int S0x[3], S1x[3], S0z[3], S1z[3];
    hat3(X0 - bx * kQOne, S0x[0], S0x[1], S0x[2]);
    hat3(X1 - bx * kQOne, S1x[0], S1x[1], S1x[2]);
    hat3(Z0 - bz * kQOne, S0z[0], S0z[1], S0z[2]);
    hat3(Z1 - bz * kQOne, S1z[0], S1z[1], S1z[2]);
    const long long sg = jsign;
    for (int b = 0; b < 3; b++) {
        const size_t row = (size_t)(bz + b) * nx;
        if (jsign != 0) {
            const long long wz = (long long)(S0z[b] + S1z[b]);
            long long acc = 0;
            for (int c = 0; c < 2; c++) {
                acc -= (long long)(S1x[c] - S0x[c]) * wz;
                if (acc != 0) atomicAdd(Jx + row + wrap_any(bx + c, nx), (u64)(sg * acc));
            }
        }
        for (int c = 0; c < 3; c++) {
            const size_t g = row + wrap_any(bx + c, nx);
            if (jsign != 0 && V != 0) {
                const long long w6 = 2LL * S0x[c] * S0z[b] + (long long)S1x[c] * S0z[b] + (long long)S0x[c] * S1z[b] +
                                     2LL * S1x[c] * S1z[b];
                if (w6 != 0) atomicAdd(Jy + g, (u64)(sg * V * w6));
            }
            if (pair) {
                const long long r = (long long)S1x[c] * S1z[b] - (long long)S0x[c] * S0z[b];
                if (r != 0) atomicAdd(rho_next + g, (u64)r);
            }
        }
    }
    if (jsign != 0) {
        for (int c = 0; c < 3; c++) {
            const long long wx = (long long)(S0x[c] + S1x[c]);
            long long acc = 0;
            for (int b = 0; b < 2; b++) {
                acc -= (long long)(S1z[b] - S0z[b]) * wx;
                if (acc != 0) atomicAdd(Jz + (size_t)(bz + b) * nx + wrap_any(bx + c, nx), (u64)(sg * acc));
            }
        }
    }
}

// Species kinds the particle code is specialised for.
enum Kind { kIon = 0, kElectron = 1, kAtom = 2 };

// One particle: state in (cell, fx, fz, ux, uy, uz) is replaced by the new state.
//   kIon:      Lorentz force + pair force, current (charge +e), node density
//   kElectron: Lorentz force, current (charge -e)
//   kAtom:     pair force, node density (neutral atoms of the transport stage)
template <int KIND, int POT>
__device__ __forceinline__ void process_particle(const StepArgs& a, const Species& S, const Window& w, int& cell,
                                                 float& fx_io, float& fz_io, float& ux, float& uy, float& uz)
{
    constexpr bool kFields = KIND != kAtom;
    constexpr bool kPair = KIND != kElectron;
    constexpr bool kCurrent = KIND != kAtom;
    constexpr int kSign = KIND == kElectron ? -1 : 1;
    const int nx = a.nx, nz = a.nz, W = w.W;
    const float fx = fx_io, fz = fz_io;
    const int cell0 = cell;
    int i, k;
    split_cell(cell0, nx, a.nx_magic, i, k);

    // window coordinates (x is periodic: take the image closest to the window centre)
    int lx = i - w.ox;
    const int centre = W / 2;
    if (lx - centre > nx / 2) lx -= nx;
    else if (centre - lx > nx / 2) lx += nx;
    const int lz = k - w.oz;
    const bool inwin = lx >= 1 && lx + 2 < W && lz >= 1 && lz + 2 < W;

    float kx = 0.f, ky = 0.f, kz = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    float n = 0.f, dnx = 0.f, dnz = 0.f;
    if (inwin) {
        const int base = lz * W + lx;
        const float gx = 1.0f - fx, gz = 1.0f - fz;
        if (kFields) {
            // four stagger patterns: (0,0) Ey, n; (1/2,0) Ex, Bz; (0,1/2) Ez, Bx; (1/2,1/2) By
            const bool ux_ = fx >= 0.5f, uz_ = fz >= 0.5f;
            const int ox_ = ux_ ? 0 : -1, oz_ = uz_ ? 0 : -W;
            const float hx = ux_ ? fx - 0.5f : fx + 0.5f, hz = uz_ ? fz - 0.5f : fz + 0.5f;
            const float ghx = 1.0f - hx, ghz = 1.0f - hz;
            // the two components of a stagger pair share their weights: one packed FP32x2 bilinear
            // sum interpolates both. Every operation here is an explicit intrinsic (no contraction
            // left to the compiler), so the single and the batched kernel round alike.
            const float2 gx2 = make_float2(gx, gx), fx2 = make_float2(fx, fx);
            const float2 gz2 = make_float2(gz, gz), fz2 = make_float2(fz, fz);
            {
                const float2* q = w.eyn + base;
                const float2 c00 = q[0], c10 = q[1], c01 = q[W], c11 = q[W + 1];
                if (kPair) {
                    const float2 r = bilerp2(c00, c10, c01, c11, gx2, fx2, gz2, fz2);
                    ky = __fmul_rn(S.e_kick, r.x);
                    n = r.y;
                    dnx = __fmaf_rn(fz, __fsub_rn(c11.y, c01.y), __fmul_rn(gz, __fsub_rn(c10.y, c00.y)));
                    dnz = __fmaf_rn(fx, __fsub_rn(c11.y, c10.y), __fmul_rn(gx, __fsub_rn(c01.y, c00.y)));
                } else {
                    ky = __fmul_rn(S.e_kick, bilerp1(c00.x, c10.x, c01.x, c11.x, gx, fx, gz, fz));
                }
            }
            {
                const float2* q = w.exbz + base + ox_;
                const float2 r = bilerp2(q[0], q[1], q[W], q[W + 1], make_float2(ghx, ghx), make_float2(hx, hx), gz2, fz2);
                kx = __fmul_rn(S.e_kick, r.x);
                bz = r.y;
            }
            {
                const float2* q = w.ezbx + base + oz_;
                const float2 r = bilerp2(q[0], q[1], q[W], q[W + 1], gx2, fx2, make_float2(ghz, ghz), make_float2(hz, hz));
                kz = __fmul_rn(S.e_kick, r.x);
                bx = r.y;
            }
            {
                const float* q = w.by + base + ox_ + oz_;
                by = bilerp1(q[0], q[1], q[W], q[W + 1], ghx, hx, ghz, hz);
            }
        } else if (kPair) {
            const float* q = w.nh + base;
            const float n00 = q[0], n10 = q[1], n01 = q[W], n11 = q[W + 1];
            n = gz * (gx * n00 + fx * n10) + fz * (gx * n01 + fx * n11);
            dnx = gz * (n10 - n00) + fz * (n11 - n01);
            dnz = gx * (n01 - n00) + fx * (n11 - n10);
        }
    } else {
        float g[9];
        gather_global(a.F[0], a.F[1], a.F[2], a.F[3], a.F[4], a.F[5], a.rho_cur, nx, nz, a.rho_s, kFields ? 1 : 0,
                      kPair ? 1 : 0, i, k, fx, fz, g);
        if (kFields) {
            kx = S.e_kick * g[0]; ky = S.e_kick * g[1]; kz = S.e_kick * g[2];
            bx = g[3]; by = g[4]; bz = g[5];
        }
        if (kPair) { n = g[6]; dnx = g[7]; dnz = g[8]; }
    }
    if (kPair) {
        float pfx, pfz;
        if (POT == kPotLJ) lj_pair_xz2(n, dnx, dnz, a.h_coef, pfx, pfz);
        else pair_force_xz<false, POT>(n, dnx, dnz, a.h_coef, a.pot_mode, a.c_att, a.s_rep, pfx, pfz, a.eam);
        kx += S.p_kick * pfx;
        kz += S.p_kick * pfz;
    }
    const float ux0 = ux, uy0 = uy, uz0 = uz;
    // relativistic Boris: half kick, rotation, half kick
    ux += kx; uy += ky; uz += kz;
    if (kFields) {
        const float rot = S.b_rot * rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        const float tx = rot * bx, ty = rot * by, tz = rot * bz;
        const float s = 2.0f * fast_rcp(1.0f + tx * tx + ty * ty + tz * tz);
        const float px = ux + (uy * tz - uz * ty);
        const float py = uy + (uz * tx - ux * tz);
        const float pz = uz + (ux * ty - uy * tx);
        ux += s * (py * tz - pz * ty);
        uy += s * (pz * tx - px * tz);
        uz += s * (px * ty - py * tx);
    }
    ux += kx; uy += ky; uz += kz;

    // move (in-plane), cells per step = u c dt / (gamma dx)
    const float step = a.cdt_dx * rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
    float dxi = ux * step, dze = uz * step;
    if (!(fabsf(dxi) < 1.0f && fabsf(dze) < 1.0f)) {
        atomicOr(a.status, (isfinite(ux) && isfinite(uy) && isfinite(uz)) ? kErrMove : kErrNan);
        ux = ux0; uy = uy0; uz = uz0; dxi = 0.0f; dze = 0.0f;
    }
    float nfx = fx + dxi;
    int di = (int)floorf(nfx);
    nfx -= (float)di;
    if (nfx >= 1.0f) { nfx = 0.0f; di += 1; }
    float nfz = fz + dze;
    int dk = 0;
    if (k == 0 && nfz < 0.0f) {                   // reflect off the wall z = 0
        nfz = -nfz; uz = -uz;
    } else if (k == nz - 1 && nfz >= 1.0f) {      // reflect off the wall z = nz
        nfz = 2.0f - nfz; uz = -uz;
    } else {
        dk = (int)floorf(nfz);
        nfz -= (float)dk;
        if (nfz >= 1.0f) { nfz = 0.0f; dk += 1; }
    }
    cell = (k + dk) * nx + wrap_x(i + di, nx);
    fx_io = nfx;
    fz_io = nfz;

    const int x0 = qoff(fx), x1 = qoff(nfx), z0 = qoff(fz), z1 = qoff(nfz);
    // |u_y| < 2^-(b+1) gives |beta_y| 2^b < 1/2, i.e. V = 0 without evaluating the code
    const int V = (kCurrent && fabsf(uy) >= a.jy_zero) ? kSign * jy_code(ux, uy, uz, a.jy_scale) : 0;
    const bool incell = inwin && (di | dk) == 0;
    if (KIND == kElectron && incell) {
        // an electron that stays in its cell (almost every electron): it always moves in fixed
        // point and almost always has V != 0, so the eight reductions onto the cell's corners are
        // issued without per-term tests (a zero term adds nothing). The out-of-plane weights are
        // 6 W = A0 U0 + A1 U1 with A = 2^16 - x and U0 = 2 C0 + C1, U1 = C0 + 2 C1 (C = 2^16 - z)
        // on the lower-left corner, and likewise with x for A and z for C on the others: two
        // widening 32 x 32-bit products per corner.
        const int d1 = i + 1 == nx ? 1 - nx : 1;
        u64* jx = a.J[0] + cell0;
        u64* jy = a.J[1] + cell0;
        u64* jz = a.J[2] + cell0;
        const int dX = x0 - x1, dZ = z0 - z1;          // charge sign -1
        atomicAdd(jx, (u64)((long long)dX * (2 * kQOne - z0 - z1)));
        atomicAdd(jx + nx, (u64)((long long)dX * (z0 + z1)));
        atomicAdd(jz, (u64)((long long)dZ * (2 * kQOne - x0 - x1)));
        atomicAdd(jz + d1, (u64)((long long)dZ * (x0 + x1)));
        const int A0 = kQOne - x0, A1 = kQOne - x1, C0 = kQOne - z0, C1 = kQOne - z1;
        const int U0 = 2 * C0 + C1, U1 = C0 + 2 * C1, Z0 = 2 * z0 + z1, Z1 = z0 + 2 * z1;
        const long long w00 = (long long)A0 * U0 + (long long)A1 * U1;
        const long long w10 = (long long)x0 * U0 + (long long)x1 * U1;
        const long long w01 = (long long)A0 * Z0 + (long long)A1 * Z1;
        const long long w11 = (long long)x0 * Z0 + (long long)x1 * Z1;
        atomicAdd(jy, (u64)(V * w00));
        atomicAdd(jy + d1, (u64)(V * w10));
        atomicAdd(jy + nx, (u64)(V * w01));
        atomicAdd(jy + nx + d1, (u64)(V * w11));
        return;
    }
    const bool moved = (di | dk) != 0 || x1 != x0 || z1 != z0;
    if (!moved && V == 0) return;                 // nothing to deposit (most ions)

    if (incell) {
        // the particle stays in its cell: stencil = the four corners of the cell (global reductions)
        const int d1 = i + 1 == nx ? 1 - nx : 1;
        if (kCurrent) {
            const int dX = kSign * (x1 - x0), dZ = kSign * (z1 - z0);
            if (dX != 0) {
                red64g(a.J[0] + cell0, (long long)dX * (2 * kQOne - z0 - z1));
                red64g(a.J[0] + cell0 + nx, (long long)dX * (z0 + z1));
            }
            if (dZ != 0) {
                red64g(a.J[2] + cell0, (long long)dZ * (2 * kQOne - x0 - x1));
                red64g(a.J[2] + cell0 + d1, (long long)dZ * (x0 + x1));
            }
            if (V != 0) {
                const int A0 = kQOne - x0, A1 = kQOne - x1, C0 = kQOne - z0, C1 = kQOne - z1;
                const int U0 = 2 * C0 + C1, U1 = C0 + 2 * C1, Z0 = 2 * z0 + z1, Z1 = z0 + 2 * z1;
                u64* jy = a.J[1] + cell0;
                red64g(jy, V * ((long long)A0 * U0 + (long long)A1 * U1));
                red64g(jy + d1, V * ((long long)x0 * U0 + (long long)x1 * U1));
                red64g(jy + nx, V * ((long long)A0 * Z0 + (long long)A1 * Z1));
                red64g(jy + nx + d1, V * ((long long)x0 * Z0 + (long long)x1 * Z1));
            }
        }
        if (kPair && moved) {
            // weights are at most 2^16: each product is one 32 x 32 -> 64-bit multiply
            const int a0 = kQOne - x0, a1 = kQOne - x1, c0 = kQOne - z0, c1 = kQOne - z1;
            u64* r = a.rho_next + cell0;
            red64g(r, (long long)a1 * c1 - (long long)a0 * c0);
            red64g(r + d1, (long long)x1 * c1 - (long long)x0 * c0);
            red64g(r + nx, (long long)a1 * z1 - (long long)a0 * z0);
            red64g(r + nx + d1, (long long)x1 * z1 - (long long)x0 * z0);
        }
    } else {
        // deposit_global applies the charge sign itself: hand it the unsigned code kSign * V
        deposit_global(a.rho_next, a.J[0], a.J[1], a.J[2], nx, i * kQOne + x0, k * kQOne + z0,
                       (i + di) * kQOne + x1, (k + dk) * kQOne + z1, kCurrent ? kSign : 0, kSign * V, kPair ? 1 : 0);
    }
}

// Part `sub` of `nsub` of one tile of one simulation: stage the tile's window, then advance that
// part of each species' particles of the tile in storage order (tiles holding many particles are
// split over several CTAs when the tiles are fewer than the CTA slots).
__device__ __forceinline__ int part_start(int p0, int p1, int sub, int nsub)
{
    return p0 + (int)(((long long)(p1 - p0) * sub) / nsub);
}

template <bool FULL, int POT>
__device__ __forceinline__ void run_tile(const StepArgs& a, int t, int sub, int nsub)
{
    extern __shared__ unsigned smem[];
    const int W = a.W, WW = W * W;
    Window w;
    w.W = W;
    float* fbase = reinterpret_cast<float*>(smem);
    w.exbz = reinterpret_cast<float2*>(fbase);
    w.ezbx = reinterpret_cast<float2*>(fbase + 2 * WW);
    w.eyn = reinterpret_cast<float2*>(fbase + 4 * WW);
    w.by = fbase + 6 * WW;
    w.nh = fbase;

    {
        int cnt = 0;
#pragma unroll
        for (int s = 0; s < 2; s++)
            if (s < a.nsp) {
                const int p0 = a.sp[s].tile_start[t], p1 = a.sp[s].tile_start[t + 1];
                cnt += part_start(p0, p1, sub + 1, nsub) - part_start(p0, p1, sub, nsub);
            }
        if (cnt == 0) return;
        const int tx = t % a.ntx, tz = t / a.ntx;
        w.ox = tx * a.T - kMargin - 1;
        w.oz = tz * a.T - kMargin - 1;
        // stage the window: fields, pair density (wall rows doubled)
        for (int j = threadIdx.x; j < WW; j += blockDim.x) {
            const int b = j / W, c = j - b * W;
            const int gx = wrap_any(w.ox + c, a.nx);
            const int gz = w.oz + b;
            const int gn = min(max(gz, 0), a.nz);          // node rows 0..nz
            const int gh = min(max(gz, 0), a.nz - 1);      // half rows 0..nz-1 (edge rows repeat)
            const size_t in = (size_t)gn * a.nx + gx, ih = (size_t)gh * a.nx + gx;
            const long long r = (long long)__ldg(a.rho_cur + in);
            const float nh = a.rho_s * (float)((gn == 0 || gn == a.nz) ? 2 * r : r);
            if (FULL) {
                w.exbz[j] = make_float2(__ldg(a.F[0] + in), __ldg(a.F[5] + in));
                w.ezbx[j] = make_float2(__ldg(a.F[2] + ih), __ldg(a.F[3] + ih));
                w.eyn[j] = make_float2(__ldg(a.F[1] + in), nh);
                w.by[j] = __ldg(a.F[4] + ih);
            } else {
                w.nh[j] = nh;
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 2; s++) {
            if (s >= a.nsp) break;
            const Species& S = a.sp[s];
            const int q0 = S.tile_start[t], q1 = S.tile_start[t + 1];
            const int p0 = part_start(q0, q1, sub, nsub), p1 = part_start(q0, q1, sub + 1, nsub);
            // the next record's position is loaded one iteration ahead (its first use is at the top
            // of the iteration); the momenta, first used after the gathers, are loaded in the iteration
            int ncell = 0;
            float nfx = 0.0f, nfz = 0.0f;
            if (p0 + (int)threadIdx.x < p1) {
                const int q = p0 + (int)threadIdx.x;
                ncell = S.a.cell[q];
                nfx = S.a.fx[q];
                nfz = S.a.fz[q];
            }
            for (int p = p0 + (int)threadIdx.x; p < p1; p += kBlock) {
                int cell = ncell;
                float fx = nfx, fz = nfz, ux = S.a.ux[p], uy = S.a.uy[p], uz = S.a.uz[p];
                if (p + kBlock < p1) {
                    ncell = S.a.cell[p + kBlock];
                    nfx = S.a.fx[p + kBlock];
                    nfz = S.a.fz[p + kBlock];
                }
                if (s == 0) process_particle<FULL ? kIon : kAtom, POT>(a, S, w, cell, fx, fz, ux, uy, uz);
                else process_particle<kElectron, POT>(a, S, w, cell, fx, fz, ux, uy, uz);
                S.a.cell[p] = cell;
                S.a.fx[p] = fx;
                S.a.fz[p] = fz;
                S.a.ux[p] = ux;
                S.a.uy[p] = uy;
                S.a.uz[p] = uz;
            }
        }
        __syncthreads();
    }
}

// Work items (a tile, or a part of a tile) are handed out dynamically: each CTA draws the next one
// from a ticket counter in the status words (measured against a static round robin: 2.034 ->
// 1.899 ms per launch on the 2048^2 slab, whose occupied tiles do not divide evenly over the
// CTAs). atomicInc wraps the counter to 0 after total + gridDim.x tickets, i.e. exactly when every
// CTA has drawn its last (failing) ticket, so every launch finds it at 0.
__device__ __forceinline__ int next_item(unsigned* ticket, int total, int* slot)
{
    if (threadIdx.x == 0) *slot = (int)atomicInc(ticket, (unsigned)(total + gridDim.x - 1));
    __syncthreads();
    const int g = *slot;
    __syncthreads();
    return g;
}

template <bool FULL, int POT>
__global__ void __launch_bounds__(kBlock, kCtasPerSm) k_particles(const StepArgs a, int nsub)
{
    __shared__ int slot;
    const int total = a.ntiles * nsub;
    for (int g = next_item(a.status + 2, total, &slot); g < total; g = next_item(a.status + 2, total, &slot))
        run_tile<FULL, POT>(a, g / nsub, g % nsub, nsub);
}

// Arguments of the simulations of a batch for the current step, in constant memory: the slab
// index is uniform across a CTA, so the kernel reads them as constant-bank operands like the
// single-simulation kernel reads its parameters. Uploaded (device to device) in front of each
// batched launch; two batches stepping at the same time on different streams would race on it.
constexpr int kMaxBatchSlabs = 48;
__constant__ StepArgs c_batch_args[kMaxBatchSlabs];
__constant__ int c_tile_base[kMaxBatchSlabs + 1];

// All simulations of a batch in one persistent launch: the tiles of every simulation form one
// work list (c_tile_base[s] = first global tile of simulation s).
template <bool FULL, int POT>
__global__ void __launch_bounds__(kBlock, kCtasPerSmBatch) k_particles_batch(int nslab, int total, int nsub)
{
    // one ticket counter for the whole batch: the first simulation's
    __shared__ int slot;
    unsigned* ticket = c_batch_args[0].status + 2;
    for (int g = next_item(ticket, total * nsub, &slot); g < total * nsub; g = next_item(ticket, total * nsub, &slot)) {
        const int tile = g / nsub;
        int s = 0;
        while (s + 1 < nslab && c_tile_base[s + 1] <= tile) s++;
        run_tile<FULL, POT>(c_batch_args[s], tile - c_tile_base[s], g % nsub, nsub);
    }
}

// parts per tile: about four work items per CTA slot (a slab often fills under half of the tiles)
static int parts_per_tile(int ntiles, int slots)
{
    int nsub = (4 * slots + ntiles - 1) / (ntiles > 0 ? ntiles : 1);
    return nsub < 1 ? 1 : (nsub > 16 ? 16 : nsub);
}

size_t particle_smem_bytes(int W) { return sizeof(unsigned) * (size_t)7 * W * W; }

// The kernel instances: Eq. (3), the altered potential and the Morse form, on the cubic and the
// HCP lattice, and the embedded-atom form on the cubic lattice (potential code in bits 0-1,
// kLatHcp in bit 2), with and without fields.
#define GBPIC_FOR_EACH_POT(X) X(kPotLJ) X(kPotAlt) X(kPotMorse) X(kPotEam) X(kPotLJ | kLatHcp) X(kPotAlt | kLatHcp) \
    X(kPotMorse | kLatHcp)

static void set_smem(const void* k, size_t shmem)
{
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    // the largest carve-out, so that several CTAs fit on one SM
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

void launch_particle_step(Ctx& c, const StepArgs& a, cudaStream_t st)
{
    const size_t shmem = particle_smem_bytes(a.W);
    // the attributes are per device: remember what each device has been given
    static std::atomic<size_t> configured[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    if (shmem > configured[dev].load()) {
#define GBPIC_ATTR(P) set_smem((const void*)k_particles<true, (P)>, shmem); set_smem((const void*)k_particles<false, (P)>, shmem);
        GBPIC_FOR_EACH_POT(GBPIC_ATTR)
#undef GBPIC_ATTR
        configured[dev].store(shmem);
    }
    const int cap = c.nsm * kCtasPerSm;
    const int nsub = parts_per_tile(a.ntiles, cap);
    int grid = a.ntiles * nsub;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    // the instance with the potential and the lattice compiled in
    switch ((a.pot_mode & 7) | (a.full ? 8 : 0)) {
#define GBPIC_CASE(P)                                                                                 \
    case 8 | (P): k_particles<true, (P)><<<grid, kBlock, shmem, st>>>(a, nsub); break;                \
    case (P): k_particles<false, (P)><<<grid, kBlock, shmem, st>>>(a, nsub); break;
        GBPIC_FOR_EACH_POT(GBPIC_CASE)
#undef GBPIC_CASE
    }
}

int max_batch_slabs() { return kMaxBatchSlabs; }

void launch_particle_step_batch(const StepArgs* args_dev, const int* tile_base_dev, int nslab, int total_tiles,
                                int full, int pot, int maxW, int nsm, cudaStream_t st)
{
    cudaMemcpyToSymbolAsync(c_batch_args, args_dev, sizeof(StepArgs) * nslab, 0, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyToSymbolAsync(c_tile_base, tile_base_dev, sizeof(int) * (nslab + 1), 0, cudaMemcpyDeviceToDevice, st);
    const size_t shmem = particle_smem_bytes(maxW);
    // the attributes are per device: remember what each device has been given
    static std::atomic<size_t> configured[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    if (shmem > configured[dev].load()) {
#define GBPIC_ATTR(P) set_smem((const void*)k_particles_batch<true, (P)>, shmem); set_smem((const void*)k_particles_batch<false, (P)>, shmem);
        GBPIC_FOR_EACH_POT(GBPIC_ATTR)
#undef GBPIC_ATTR
        configured[dev].store(shmem);
    }
    const int cap = nsm * kCtasPerSmBatch;
    const int nsub = parts_per_tile(total_tiles, cap);
    int grid = total_tiles * nsub < cap ? total_tiles * nsub : cap;
    if (grid < 1) grid = 1;
    // pot: the instance code shared by every slab (potential and lattice)
    switch ((pot & 7) | (full ? 8 : 0)) {
#define GBPIC_CASE(P)                                                                                          \
    case 8 | (P): k_particles_batch<true, (P)><<<grid, kBlock, shmem, st>>>(nslab, total_tiles, nsub); break;   \
    case (P): k_particles_batch<false, (P)><<<grid, kBlock, shmem, st>>>(nslab, total_tiles, nsub); break;
        GBPIC_FOR_EACH_POT(GBPIC_CASE)
#undef GBPIC_CASE
    }
}

int tile_window(int T) { return T + 2 * kMargin + 3; }

}  // namespace gbpic
