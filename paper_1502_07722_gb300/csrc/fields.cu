// Maxwell update of the PIC cycle (paper: PIC integrates the Maxwell and Lorentz equations),
// 2D3V Yee scheme with d/dy = 0: B advanced by half a step, E by a full step with the current
// of the particle kernel (int64 fixed point -> A/m^2) and the laser antenna, B by the second
// half step. x is periodic; the tangential E components on the wall rows z = 0 and z = nz take
// the first-order Mur absorbing condition.
#include "pic_internal.cuh"

namespace gbpic {

struct FieldArgs {
    int nx, nz, k_ant;
    float h_b;           // dt / (2 dx)      (half step of B)
    float h_e;           // c^2 dt / dx      (full step of E)
    float cj;            // J2x, J2z -> dt J / eps0
    float cjy;           // J6y -> dt J_y / eps0
    float mur;           // (c dt - dx) / (c dt + dx)
    float ant_s, ant_c;  // antenna amplitude at this step: E_x += ant_c(x) * ant_s + ant_s(x) * ant_c
    float* F[6];
    const u64* J[3];
    float* save;         // 8 * nx: Ex(0) Ex(1) Ex(nz-1) Ex(nz) Ey(0) Ey(1) Ey(nz-1) Ey(nz) before the E step
    const float* antc;
    const float* ants;
};

__global__ void k_half_B(const FieldArgs f, int save)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= f.nx) return;
    const int nx = f.nx, nz = f.nz;
    const int ip = i + 1 == nx ? 0 : i + 1;
    const size_t c = (size_t)k * nx + i;
    const float *Ex = f.F[0], *Ey = f.F[1], *Ez = f.F[2];
    float *Bx = f.F[3], *By = f.F[4], *Bz = f.F[5];
    const float ey = Ey[c];
    if (k < nz) {
        const size_t u = c + nx;
        Bx[c] += f.h_b * (Ey[u] - ey);
        By[c] += f.h_b * ((Ez[(size_t)k * nx + ip] - Ez[c]) - (Ex[u] - Ex[c]));
    }
    Bz[c] -= f.h_b * (Ey[(size_t)k * nx + ip] - ey);
    if (save) {
        int slot = -1;
        if (k == 0) slot = 0;
        else if (k == 1) slot = 1;
        else if (k == nz - 1) slot = 2;
        else if (k == nz) slot = 3;
        if (slot >= 0) {
            f.save[slot * nx + i] = Ex[c];
            f.save[(4 + slot) * nx + i] = ey;
        }
    }
}

// new Ex / Ey of an interior node (i, k) from its old value
__device__ __forceinline__ float ex_new(const FieldArgs& f, int i, int k, float old)
{
    const size_t c = (size_t)k * f.nx + i;
    float v = old - f.h_e * (f.F[4][c] - f.F[4][c - f.nx]) - f.cj * (float)(long long)f.J[0][c];
    if (k == f.k_ant) v += f.antc[i] * f.ant_s + f.ants[i] * f.ant_c;
    return v;
}
__device__ __forceinline__ float ey_new(const FieldArgs& f, int i, int k, float old)
{
    const size_t c = (size_t)k * f.nx + i;
    const int im = i == 0 ? f.nx - 1 : i - 1;
    return old + f.h_e * ((f.F[3][c] - f.F[3][c - f.nx]) - (f.F[5][c] - f.F[5][(size_t)k * f.nx + im])) -
           f.cjy * (float)(long long)f.J[1][c];
}

__global__ void k_E(const FieldArgs f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= f.nx) return;
    const int nx = f.nx, nz = f.nz;
    const size_t c = (size_t)k * nx + i;
    float* Ex = f.F[0];
    float* Ey = f.F[1];
    float* Ez = f.F[2];
    if (k > 0 && k < nz) {
        Ex[c] = ex_new(f, i, k, Ex[c]);
        Ey[c] = ey_new(f, i, k, Ey[c]);
    } else if (k == 0) {
        const float x0 = f.save[0 * nx + i], x1 = f.save[1 * nx + i];
        const float y0 = f.save[4 * nx + i], y1 = f.save[5 * nx + i];
        Ex[c] = x1 + f.mur * (ex_new(f, i, 1, x1) - x0);
        Ey[c] = y1 + f.mur * (ey_new(f, i, 1, y1) - y0);
    } else {
        const float x1 = f.save[2 * nx + i], x0 = f.save[3 * nx + i];
        const float y1 = f.save[6 * nx + i], y0 = f.save[7 * nx + i];
        Ex[c] = x1 + f.mur * (ex_new(f, i, nz - 1, x1) - x0);
        Ey[c] = y1 + f.mur * (ey_new(f, i, nz - 1, y1) - y0);
    }
    if (k < nz) {
        const int im = i == 0 ? nx - 1 : i - 1;
        Ez[c] += f.h_e * (f.F[4][c] - f.F[4][(size_t)k * nx + im]) - f.cj * (float)(long long)f.J[2][c];
    }
}

void launch_fields(Ctx& c, cudaStream_t st, double t_half, int64_t* launches)
{
    FieldArgs f;
    f.nx = c.nx;
    f.nz = c.nz;
    f.k_ant = c.k_ant;
    f.h_b = (float)(0.5 * c.dt / c.cfg.dx);
    f.h_e = (float)(kC * kC * c.dt / c.cfg.dx);
    f.cj = (float)(kQe * c.w / (8589934592.0 * c.cfg.dx * kEps0));
    f.cjy = (float)(kQe * c.w * kC * c.dt / (6.0 * 1125899906842624.0 * c.cfg.dx * c.cfg.dx * kEps0));
    const double cdt = kC * c.dt;
    f.mur = (float)((cdt - c.cfg.dx) / (cdt + c.cfg.dx));
    // antenna: E_x += 2 (c dt / dx) E0 env(t) amp(x) sin(w (t - t_ant) + phi(x))
    double ant_s = 0.0, ant_c = 0.0;
    if (c.cfg.laser_profile != PIC_LASER_NONE) {
        const double tau = t_half - c.t_ant;
        const double env = exp(-2.0 * log(2.0) * tau * tau / (c.cfg.tau_fwhm * c.cfg.tau_fwhm));
        const double a = 2.0 * (cdt / c.cfg.dx) * c.E0 * env;
        ant_s = a * sin(c.omega * tau);
        ant_c = a * cos(c.omega * tau);
    }
    f.ant_s = (float)ant_s;
    f.ant_c = (float)ant_c;
    for (int q = 0; q < 6; q++) f.F[q] = c.F[q];
    for (int q = 0; q < 3; q++) f.J[q] = c.J[q];
    f.save = c.mur_save;
    f.antc = c.ant_c;
    f.ants = c.ant_s;
    dim3 block(256);
    dim3 grid((c.nx + 255) / 256, c.nz + 1);
    k_half_B<<<grid, block, 0, st>>>(f, 1);
    k_E<<<grid, block, 0, st>>>(f);
    k_half_B<<<grid, block, 0, st>>>(f, 0);
    if (launches) *launches += 3;
}

}  // namespace gbpic
