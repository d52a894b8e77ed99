// The particle kernel of one PIC step (paper, the PIC-cycle paragraph and Fig. 1B):
// for every macroparticle -- gather E, B (Lorentz force) and the node density with its gradient
// (pair-potential force, Eqs. 1-3) -> relativistic Boris push -> move -> charge-conserving
// current deposition (Esirkepov, fixed point) -> node density at the new position.
//
// One CTA owns one tile of T x T cells at a time (particles are sorted into tiles). The
// deposits of a tile go into int64 accumulators in shared memory that cover the tile plus a
// margin, and are flushed to global memory with one atomic per non-zero node. Particles that
// drifted beyond the margin since the last sort deposit straight into global memory. Integer
// sums make the result independent of the order of the atomics.
#include "pic_device.cuh"

namespace gbpic {

constexpr int kMargin = 2;          // cells a particle may drift out of its tile between sorts
constexpr int kBlock = 256;

__device__ __forceinline__ int wrap_any(int i, int nx)
{
    int r = i % nx;
    return r < 0 ? r + nx : r;
}

__device__ __forceinline__ void dep(bool local, u64* s, u64* g, int W, int nx, int lb, int la, int gb, int ga,
                                    long long v)
{
    if (v == 0) return;
    if (local) atomicAdd(s + lb * W + la, (u64)v);
    else atomicAdd(g + (size_t)gb * nx + wrap_any(ga, nx), (u64)v);
}

template <bool FULL>
__device__ __forceinline__ void process_particle(const StepArgs& a, const Species& S, int p, u64* s_rho, u64* s_jx,
                                                 u64* s_jy, u64* s_jz, int ox, int oz)
{
    const int nx = a.nx, nz = a.nz, W = a.W;
    const int cell = S.a.cell[p];
    const float fx = S.a.fx[p], fz = S.a.fz[p];
    float ux = S.a.ux[p], uy = S.a.uy[p], uz = S.a.uz[p];
    const int k = cell / nx, i = cell - k * nx;

    // half kick (electric + pair force), rotation field
    float kx = 0.f, ky = 0.f, kz = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    if (FULL) {
        kx = S.e_kick * gather_field(a.F[0], nx, nz, i, k, fx, fz, 1, 0);
        ky = S.e_kick * gather_field(a.F[1], nx, nz, i, k, fx, fz, 0, 0);
        kz = S.e_kick * gather_field(a.F[2], nx, nz, i, k, fx, fz, 0, 1);
        bx = gather_field(a.F[3], nx, nz, i, k, fx, fz, 0, 1);
        by = gather_field(a.F[4], nx, nz, i, k, fx, fz, 1, 1);
        bz = gather_field(a.F[5], nx, nz, i, k, fx, fz, 1, 0);
    }
    if (S.pair) {
        float n, dnx, dnz;
        gather_density(a.rho_cur, nx, nz, a.rho_s, i, k, fx, fz, n, dnx, dnz);
        if (n > 0.0f) {
            float c = cbrtf(n);
            float inv43 = 1.0f / (n * c);
            kx += S.p_kick * pair_axis(n, c, inv43, dnx, a.h_coef, a.pot_mode, a.c_att, a.s_rep);
            kz += S.p_kick * pair_axis(n, c, inv43, dnz, a.h_coef, a.pot_mode, a.c_att, a.s_rep);
        }
    }
    const float ux0 = ux, uy0 = uy, uz0 = uz;
    // relativistic Boris: half kick, rotation, half kick
    ux += kx; uy += ky; uz += kz;
    if (FULL) {
        float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        float tx = S.b_rot * ig * bx, ty = S.b_rot * ig * by, tz = S.b_rot * ig * bz;
        float s = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
        float px = ux + (uy * tz - uz * ty);
        float py = uy + (uz * tx - ux * tz);
        float pz = uz + (ux * ty - uy * tx);
        ux += s * (py * tz - pz * ty);
        uy += s * (pz * tx - px * tz);
        uz += s * (px * ty - py * tx);
    }
    ux += kx; uy += ky; uz += kz;

    // move (in-plane), cells per step = u c dt / (gamma dx)
    float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
    float dxi = ux * a.cdt_dx * ig, dze = uz * a.cdt_dx * ig;
    if (!(fabsf(dxi) < 1.0f && fabsf(dze) < 1.0f)) {
        atomicOr(a.status, (isfinite(ux) && isfinite(uy) && isfinite(uz)) ? kErrMove : kErrNan);
        ux = ux0; uy = uy0; uz = uz0; dxi = 0.0f; dze = 0.0f;
    }
    float nfx = fx + dxi;
    int di = (int)floorf(nfx);
    nfx -= (float)di;
    if (nfx >= 1.0f) { nfx = 0.0f; di += 1; }
    float nfz = fz + dze;
    int k1 = k;
    if (k == 0 && nfz < 0.0f) {                   // reflect off the wall z = 0
        nfz = -nfz; uz = -uz;
    } else if (k == nz - 1 && nfz >= 1.0f) {      // reflect off the wall z = nz
        nfz = 2.0f - nfz; uz = -uz;
    } else {
        int dk = (int)floorf(nfz);
        nfz -= (float)dk;
        if (nfz >= 1.0f) { nfz = 0.0f; dk += 1; }
        k1 = k + dk;
    }
    const int i1u = i + di;
    const int i1 = wrap_x(i1u, nx);

    // fixed-point coordinates relative to the tile window
    int lx0 = i - ox;
    const int centre = W / 2;
    if (lx0 - centre > nx / 2) lx0 -= nx;
    else if (centre - lx0 > nx / 2) lx0 += nx;
    const int XL0 = lx0 * kQOne + qoff(fx);
    const int XL1 = XL0 + (i1u - i) * kQOne + qoff(nfx) - qoff(fx);
    const int ZL0 = (k - oz) * kQOne + qoff(fz);
    const int ZL1 = ZL0 + (k1 - k) * kQOne + qoff(nfz) - qoff(fz);
    const int bxl = min(XL0, XL1) >> kQBits;
    const int bzl = min(ZL0, ZL1) >> kQBits;
    const bool local = bxl >= 0 && bxl + 2 < W && bzl >= 0 && bzl + 2 < W;
    const int gbx = bxl + ox, gbz = bzl + oz;
    int S0x[3], S1x[3], S0z[3], S1z[3];
    hat3(XL0 - bxl * kQOne, S0x[0], S0x[1], S0x[2]);
    hat3(XL1 - bxl * kQOne, S1x[0], S1x[1], S1x[2]);
    hat3(ZL0 - bzl * kQOne, S0z[0], S0z[1], S0z[2]);
    hat3(ZL1 - bzl * kQOne, S1z[0], S1z[1], S1z[2]);

    if (S.jsign != 0) {
        const long long sg = S.jsign;
#pragma unroll
        for (int b = 0; b < 3; b++) {                       // J_x on node row b
            long long wz = (long long)(S0z[b] + S1z[b]);
            if (wz == 0) continue;
            long long acc = -(long long)(S1x[0] - S0x[0]) * wz;
            dep(local, s_jx, a.J[0], W, nx, bzl + b, bxl, gbz + b, gbx, sg * acc);
            acc -= (long long)(S1x[1] - S0x[1]) * wz;
            dep(local, s_jx, a.J[0], W, nx, bzl + b, bxl + 1, gbz + b, gbx + 1, sg * acc);
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {                       // J_z on node column c
            long long wx = (long long)(S0x[c] + S1x[c]);
            if (wx == 0) continue;
            long long acc = -(long long)(S1z[0] - S0z[0]) * wx;
            dep(local, s_jz, a.J[2], W, nx, bzl, bxl + c, gbz, gbx + c, sg * acc);
            acc -= (long long)(S1z[1] - S0z[1]) * wx;
            dep(local, s_jz, a.J[2], W, nx, bzl + 1, bxl + c, gbz + 1, gbx + c, sg * acc);
        }
        const int V = jy_code(ux, uy, uz);
        if (V != 0) {
            const long long sv = sg * (long long)V;
#pragma unroll
            for (int b = 0; b < 3; b++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    long long w6 = 2LL * S0x[c] * S0z[b] + (long long)S1x[c] * S0z[b] + (long long)S0x[c] * S1z[b] +
                                   2LL * S1x[c] * S1z[b];
                    dep(local, s_jy, a.J[1], W, nx, bzl + b, bxl + c, gbz + b, gbx + c, sv * w6);
                }
        }
    }
    if (S.pair) {                                           // node density at the new position
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int c = 0; c < 3; c++)
                dep(local, s_rho, a.rho_next, W, nx, bzl + b, bxl + c, gbz + b, gbx + c,
                    (long long)S1x[c] * S1z[b]);
    }

    S.a.cell[p] = k1 * nx + i1;
    S.a.fx[p] = nfx;
    S.a.fz[p] = nfz;
    S.a.ux[p] = ux;
    S.a.uy[p] = uy;
    S.a.uz[p] = uz;
}

template <bool FULL>
__global__ void __launch_bounds__(kBlock) k_particles(const StepArgs a)
{
    extern __shared__ u64 smem[];
    const int W = a.W, WW = W * W;
    u64* s_rho = smem;
    u64* s_jx = smem + WW;
    u64* s_jy = smem + 2 * WW;
    u64* s_jz = smem + 3 * WW;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        int cnt = 0;
#pragma unroll
        for (int s = 0; s < 2; s++)
            if (s < a.nsp) cnt += a.sp[s].tile_start[t + 1] - a.sp[s].tile_start[t];
        if (cnt == 0) continue;
        for (int j = threadIdx.x; j < 4 * WW; j += blockDim.x) smem[j] = 0;
        __syncthreads();
        const int tx = t % a.ntx, tz = t / a.ntx;
        const int ox = tx * a.T - kMargin - 1, oz = tz * a.T - kMargin - 1;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            if (s >= a.nsp) break;
            const int p0 = a.sp[s].tile_start[t], p1 = a.sp[s].tile_start[t + 1];
            for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x)
                process_particle<FULL>(a, a.sp[s], p, s_rho, s_jx, s_jy, s_jz, ox, oz);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < WW; j += blockDim.x) {
            const int b = j / W, c = j - b * W;
            const int gz = oz + b;
            if (gz < 0 || gz > a.nz) continue;
            const size_t g = (size_t)gz * a.nx + wrap_any(ox + c, a.nx);
            u64 v;
            if ((v = s_rho[j]) != 0) atomicAdd(a.rho_next + g, v);
            if ((v = s_jx[j]) != 0) atomicAdd(a.J[0] + g, v);
            if ((v = s_jy[j]) != 0) atomicAdd(a.J[1] + g, v);
            if ((v = s_jz[j]) != 0) atomicAdd(a.J[2] + g, v);
        }
        __syncthreads();
    }
}

void launch_particle_step(Ctx& c, const StepArgs& a, cudaStream_t st)
{
    const size_t shmem = 4 * sizeof(u64) * (size_t)a.W * a.W;
    static size_t configured = 0;
    if (shmem > 48 * 1024 && shmem > configured) {
        cudaFuncSetAttribute(k_particles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
        cudaFuncSetAttribute(k_particles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
        configured = shmem;
    }
    int grid = a.ntiles;
    const int cap = c.nsm * 4;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (a.full) k_particles<true><<<grid, kBlock, shmem, st>>>(a);
    else k_particles<false><<<grid, kBlock, shmem, st>>>(a);
}

int tile_window(int T) { return T + 2 * kMargin + 3; }

}  // namespace gbpic
