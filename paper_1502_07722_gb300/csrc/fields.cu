// Maxwell update of the PIC cycle (paper: PIC integrates the Maxwell and Lorentz equations),
// 2D3V Yee scheme with d/dy = 0: B advanced by half a step, E by a full step with the current
// of the particle kernel (int64 fixed point -> A/m^2) and the laser antenna, B by the second
// half step. x is periodic; the tangential E components on the wall rows z = 0 and z = nz take
// the first-order Mur absorbing condition.
//
// The same node functions serve one simulation (one launch per kernel) and a batch of
// simulations (one launch per kernel for all of them, blockIdx.z = simulation).
#include "pic_internal.cuh"

namespace gbpic {

// Antenna amplitude of one step (FP64 on the device, one thread):
//   E_x += 2 (c dt / dx) E0 env(t) amp(x) sin(w (t - t_ant) + phi(x))
// split as ant[0] * amp cos(phi) + ant[1] * amp sin(phi) with ant = A (sin, cos)(w (t - t_ant)).
__device__ __forceinline__ void antenna_scalars(const AntennaParams& p, long long step, float* ant)
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

__global__ void k_antenna(AntennaParams p, long long step, float* ant) { antenna_scalars(p, step, ant); }

// batched: slab s reads its own step counter, advances it after the step (k_step_done)
__global__ void k_antenna_batch(const AntennaParams* p, const long long* step, float* ant, int nslab)
{
    const int s = threadIdx.x;
    if (s < nslab) antenna_scalars(p[s], step[s], ant + 2 * s);
}

__global__ void k_step_done(long long* step, int nslab)
{
    const int s = threadIdx.x;
    if (s < nslab) step[s] += 1;
}

__device__ __forceinline__ void half_B_node(const FieldArgs& f, int i, int k, int save)
{
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
    if (k == f.k_ant) v += f.antc[i] * f.ant[0] + f.ants[i] * f.ant[1];
    return v;
}
__device__ __forceinline__ float ey_new(const FieldArgs& f, int i, int k, float old)
{
    const size_t c = (size_t)k * f.nx + i;
    const int im = i == 0 ? f.nx - 1 : i - 1;
    return old + f.h_e * ((f.F[3][c] - f.F[3][c - f.nx]) - (f.F[5][c] - f.F[5][(size_t)k * f.nx + im])) -
           f.cjy * (float)(long long)f.J[1][c];
}

// E update of one node; returns, on the flux row, the node's (Ex By - Ey Bx) at the half step
// (E the mean of old and new, B averaged over the half rows on either side), else 0
__device__ __forceinline__ float E_node(const FieldArgs& f, int i, int k)
{
    const int nx = f.nx, nz = f.nz;
    const size_t c = (size_t)k * nx + i;
    float* Ex = f.F[0];
    float* Ey = f.F[1];
    float* Ez = f.F[2];
    float s = 0.0f;
    if (k > 0 && k < nz) {
        const float ex0 = Ex[c], ey0 = Ey[c];
        const float ex1 = ex_new(f, i, k, ex0), ey1 = ey_new(f, i, k, ey0);
        Ex[c] = ex1;
        Ey[c] = ey1;
        if (k == f.k_flux)
            s = 0.25f * ((ex0 + ex1) * (f.F[4][c - nx] + f.F[4][c]) - (ey0 + ey1) * (f.F[3][c - nx] + f.F[3][c]));
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
    return s;
}

// the flux row's warp sums into the FP64 accumulator
__device__ __forceinline__ void add_flux(const FieldArgs& f, int k, float s)
{
    if (k != f.k_flux) return;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(f.flux, (double)s);
}

__global__ void k_half_B(const FieldArgs f, int save)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < f.nx) half_B_node(f, i, blockIdx.y, save);
}

__global__ void k_E(const FieldArgs f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float s = i < f.nx ? E_node(f, i, blockIdx.y) : 0.0f;
    add_flux(f, blockIdx.y, s);
}

// Batched field kernels: blockIdx.x runs over every slab's (row, 256-node segment) blocks, slab s
// owning blocks rb[s] .. rb[s + 1] - 1. Every slab's arguments travel in the launch's parameter
// block (a grid over the largest slab's rows for every slab, reading the arguments from global
// memory, took 0.27 ms per step of the 16-slab sweep).
__device__ __forceinline__ int batch_slab(const FieldBatch& P, int g)
{
    int s = 0;
    while (s + 1 < P.n && P.rb[s + 1] <= g) s++;
    return s;
}

__global__ void k_half_B_batch(const __grid_constant__ FieldBatch P, int save)
{
    const int s = batch_slab(P, (int)blockIdx.x);
    const FieldArgs& f = P.f[s];
    const int local = (int)blockIdx.x - P.rb[s], nxb = (f.nx + 255) >> 8;
    const int k = local / nxb, i = (local - k * nxb) * 256 + (int)threadIdx.x;
    if (i < f.nx) half_B_node(f, i, k, save);
}

__global__ void k_E_batch(const __grid_constant__ FieldBatch P)
{
    const int s = batch_slab(P, (int)blockIdx.x);
    const FieldArgs& f = P.f[s];
    const int local = (int)blockIdx.x - P.rb[s], nxb = (f.nx + 255) >> 8;
    const int k = local / nxb, i = (local - k * nxb) * 256 + (int)threadIdx.x;   // k uniform over the block
    const float v = i < f.nx ? E_node(f, i, k) : 0.0f;
    add_flux(f, k, v);
}

// each slab's first block (rb[n] = the total)
void field_row_blocks(FieldBatch& P)
{
    P.rb[0] = 0;
    for (int s = 0; s < P.n; s++) P.rb[s + 1] = P.rb[s] + (P.f[s].nz + 1) * ((P.f[s].nx + 255) / 256);
}

AntennaParams make_antenna_params(const Ctx& c)
{
    AntennaParams p;
    p.on = c.cfg.laser_profile != PIC_LASER_NONE;
    p.dt = c.dt;
    p.t_ant = c.t_ant;
    p.tau_fwhm = c.cfg.tau_fwhm > 0 ? c.cfg.tau_fwhm : 1.0;
    p.omega = c.omega;
    p.coef = 2.0 * (kC * c.dt / c.cfg.dx) * c.E0;
    return p;
}

FieldArgs make_field_args(const Ctx& c)
{
    FieldArgs f;
    f.nx = c.nx;
    f.nz = c.nz;
    f.k_ant = c.k_ant;
    f.h_b = (float)(0.5 * c.dt / c.cfg.dx);
    f.h_e = (float)(kC * kC * c.dt / c.cfg.dx);
    f.cj = (float)(kQe * c.w / (8589934592.0 * c.cfg.dx * kEps0));
    f.cjy = (float)(kQe * c.w * kC * c.dt / (6.0 * ldexp(1.0, 32 + c.jy_bits) * c.cfg.dx * c.cfg.dx * kEps0));
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
    return f;
}

void launch_fields(Ctx& c, cudaStream_t st, int64_t step, int64_t* launches)
{
    const FieldArgs f = make_field_args(c);
    k_antenna<<<1, 1, 0, st>>>(make_antenna_params(c), (long long)step, c.ant);
    dim3 block(256);
    dim3 grid((c.nx + 255) / 256, c.nz + 1);
    k_half_B<<<grid, block, 0, st>>>(f, 1);
    k_E<<<grid, block, 0, st>>>(f);
    k_half_B<<<grid, block, 0, st>>>(f, 0);
    if (launches) *launches += 4;
}

void launch_fields_batch(const FieldBatch& P, const AntennaParams* ap_dev, long long* step_dev, float* ant_dev,
                         cudaStream_t st)
{
    k_antenna_batch<<<1, 32, 0, st>>>(ap_dev, step_dev, ant_dev, P.n);
    const int blocks = P.rb[P.n];
    k_half_B_batch<<<blocks, 256, 0, st>>>(P, 1);
    k_E_batch<<<blocks, 256, 0, st>>>(P);
    k_half_B_batch<<<blocks, 256, 0, st>>>(P, 0);
    k_step_done<<<1, 32, 0, st>>>(step_dev, P.n);
}

}  // namespace gbpic
