// Stand-alone entry kernels: node density of the pair species at the current positions (paper:
// weights interpolated to the nearest surrounding nodes) and the per-atom pair force from that
// density (Eqs. 1-3), without advancing the particles.
#include "pic_device.cuh"

namespace gbpic {

__global__ void k_deposit_density(const int32_t* __restrict__ cell, const float* __restrict__ fx,
                                  const float* __restrict__ fz, int64_t n, int nx, int nz, u64* out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[p];
        const int k = c / nx, i = c - k * nx;
        const int qx = qoff(fx[p]), qz = qoff(fz[p]);
        const int i1 = i + 1 == nx ? 0 : i + 1;
        const long long sx0 = kQOne - qx, sx1 = qx, sz0 = kQOne - qz, sz1 = qz;
        const size_t r0 = (size_t)k * nx, r1 = r0 + nx;
        if (sx0 * sz0) atomicAdd(out + r0 + i, (u64)(sx0 * sz0));
        if (sx1 * sz0) atomicAdd(out + r0 + i1, (u64)(sx1 * sz0));
        if (sx0 * sz1) atomicAdd(out + r1 + i, (u64)(sx0 * sz1));
        if (sx1 * sz1) atomicAdd(out + r1 + i1, (u64)(sx1 * sz1));
    }
}

__global__ void k_pair_force(const int32_t* __restrict__ cell, const float* __restrict__ fx,
                             const float* __restrict__ fz, int64_t n, int nx, int nz, const u64* __restrict__ rho,
                             float rho_s, float h_coef, int pot_mode, float c_att, float s_rep, float f_unit,
                             EamP eam, float* __restrict__ out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[p];
        const int k = c / nx, i = c - k * nx;
        float dens, dnx, dnz;
        gather_density(rho, nx, nz, rho_s, i, k, fx[p], fz[p], dens, dnx, dnz);
        float Fx, Fz;
        pair_force_xz(dens, dnx, dnz, h_coef, pot_mode, c_att, s_rep, Fx, Fz, eam);
        out[3 * p + 0] = f_unit * Fx;
        out[3 * p + 1] = 0.0f;
        out[3 * p + 2] = f_unit * Fz;
    }
}

// Pair force at probe positions that add nothing to the density (the calibration of the attractive
// factor follows one atom out of the target). A probe outside the grid or with an offset outside
// [0, 1) x [0, 1] reads nothing and gets NaN.
__global__ void k_pair_force_probe(const int32_t* __restrict__ cell, const float* __restrict__ fx,
                                   const float* __restrict__ fz, int64_t n, int nx, int nz,
                                   const u64* __restrict__ rho, float rho_s, float h_coef, int pot_mode,
                                   float c_att, float s_rep, float f_unit, EamP eam, float* __restrict__ out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[p];
        const float a = fx[p], b = fz[p];
        if (c < 0 || c >= nx * nz || !(a >= 0.0f && a < 1.0f && b >= 0.0f && b <= 1.0f)) {
            out[3 * p + 0] = out[3 * p + 1] = out[3 * p + 2] = __int_as_float(0x7fc00000);
            continue;
        }
        const int k = c / nx, i = c - k * nx;
        float dens, dnx, dnz;
        gather_density(rho, nx, nz, rho_s, i, k, a, b, dens, dnx, dnz);
        float Fx, Fz;
        pair_force_xz<true>(dens, dnx, dnz, h_coef, pot_mode, c_att, s_rep, Fx, Fz, eam);
        out[3 * p + 0] = f_unit * Fx;
        out[3 * p + 1] = 0.0f;
        out[3 * p + 2] = f_unit * Fz;
    }
}

// Flags particles outside the grid or with offsets outside [0,1) x [0,1] (bit 0 of *bad).
__global__ void k_validate(const int32_t* __restrict__ cell, const float* __restrict__ fx,
                           const float* __restrict__ fy, const float* __restrict__ fz, int64_t n, int64_t ncell,
                           unsigned* bad)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[p];
        const float a = fx[p], b = fz[p], y = fy ? fy[p] : 0.0f;
        if (c < 0 || c >= ncell || !(a >= 0.0f && a < 1.0f && b >= 0.0f && b <= 1.0f && y >= 0.0f && y < 1.0f))
            atomicOr(bad, 1u);
    }
}

static int grid_for(const Ctx& c, int64_t n)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)c.nsm * 8;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

void launch_deposit_density(Ctx& c, u64* out, cudaStream_t st)
{
    cudaMemsetAsync(out, 0, sizeof(u64) * c.nn, st);
    const Species& S = c.sp[0];
    if (S.n == 0) return;
    k_deposit_density<<<grid_for(c, S.n), 256, 0, st>>>(S.a.cell, S.a.fx, S.a.fz, S.n, c.nx, c.nz, out);
}

void launch_validate(Ctx& c, const SpeciesBuf& b, int64_t n, unsigned* bad, cudaStream_t st)
{
    if (n == 0) return;
    k_validate<<<grid_for(c, n), 256, 0, st>>>(b.cell, b.fx, c.dims == 3 ? b.fy : nullptr, b.fz, n,
                                               (int64_t)c.nx * c.ny * c.nz, bad);
}

void launch_pair_force_probe(Ctx& c, int64_t n, const int32_t* cell, const float* fx, const float* fz, int pot_mode,
                             double c_att, double s_rep, float* out, cudaStream_t st)
{
    if (n == 0) return;
    k_pair_force_probe<<<grid_for(c, n), 256, 0, st>>>(cell, fx, fz, n, c.nx, c.nz, c.rho[c.cur], (float)c.rho_scale,
                                                      (float)(c.r0 / (6.0 * c.cfg.dx)), pot_mode, (float)c_att,
                                                      (float)s_rep, (float)(c.D / c.r0), eam_params(c.cfg), out);
}

void launch_pair_force(Ctx& c, float* out, cudaStream_t st)
{
    const Species& S = c.sp[0];
    if (S.n == 0) return;
    k_pair_force<<<grid_for(c, S.n), 256, 0, st>>>(S.a.cell, S.a.fx, S.a.fz, S.n, c.nx, c.nz, c.rho[c.cur],
                                                   (float)c.rho_scale, (float)(c.r0 / (6.0 * c.cfg.dx)),
                                                   pot_code(c.cfg), pot_param(c.cfg), (float)c.cfg.s_rep,
                                                   (float)(c.D / c.r0), eam_params(c.cfg), out);
}

}  // namespace gbpic
