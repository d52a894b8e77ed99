// Coupling of the two stages (paper: the atomic-transport run starts from the lattice temperature
// the laser-interaction run leaves once electrons and lattice have equilibrated).
//  * Lattice temperature per cell of one species: T = m c^2 / (3 k_B) sum |u - mean u|^2 / (N - 1)
//    over the N particles of the cell (the thermal spread about the cell's mean flow); cells with
//    fewer than two particles get 0. Per-cell sums in FP64 (atomics), then one thread per cell.
//  * Re-tempering to a map: momenta drawn at the uniform temperature T_from become the same draws
//    at the temperature of their cell, u -> u sqrt(T_cell / T_from).
#include "pic_internal.cuh"

namespace gbpic {

__global__ void k_cell_moments(const int32_t* __restrict__ cell, const float* __restrict__ ux,
                               const float* __restrict__ uy, const float* __restrict__ uz, int64_t n, int64_t ncell,
                               double* __restrict__ acc)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = cell[p];
        const double a = ux[p], b = uy[p], c = uz[p];
        atomicAdd(acc + q, 1.0);
        atomicAdd(acc + ncell + q, a);
        atomicAdd(acc + 2 * ncell + q, b);
        atomicAdd(acc + 3 * ncell + q, c);
        atomicAdd(acc + 4 * ncell + q, a * a + b * b + c * c);
    }
}

__global__ void k_cell_temperature(const double* __restrict__ acc, int64_t ncell, double mc2_3k, double* __restrict__ T)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ncell; q += (int64_t)gridDim.x * blockDim.x) {
        const double n = acc[q];
        if (n < 2.0) {
            T[q] = 0.0;
            continue;
        }
        const double mx = acc[ncell + q] / n, my = acc[2 * ncell + q] / n, mz = acc[3 * ncell + q] / n;
        T[q] = mc2_3k * (acc[4 * ncell + q] - n * (mx * mx + my * my + mz * mz)) / (n - 1.0);
    }
}

__global__ void k_set_temperature(const int32_t* __restrict__ cell, float* ux, float* uy, float* uz, int64_t n,
                                  const double* __restrict__ T, double T_from)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double f = sqrt(T[cell[p]] / T_from);
        ux[p] = (float)((double)ux[p] * f);
        uy[p] = (float)((double)uy[p] * f);
        uz[p] = (float)((double)uz[p] * f);
    }
}

static int grid_of(const Ctx& c, int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)c.nsm * 16) g = (int64_t)c.nsm * 16;
    return g < 1 ? 1 : (int)g;
}

void launch_cell_temperature(Ctx& c, int s, double* work, double* T, cudaStream_t st)
{
    const Species& S = c.sp[s];
    const int64_t ncell = (int64_t)c.nx * c.ny * c.nz;
    cudaMemsetAsync(work, 0, sizeof(double) * 5 * (size_t)ncell, st);
    if (S.n > 0) k_cell_moments<<<grid_of(c, S.n), 256, 0, st>>>(S.a.cell, S.a.ux, S.a.uy, S.a.uz, S.n, ncell, work);
    k_cell_temperature<<<grid_of(c, ncell), 256, 0, st>>>(work, ncell, S.mass * kC * kC / (3.0 * kKb), T);
}

void launch_set_temperature(Ctx& c, int s, const double* T, double T_from, cudaStream_t st)
{
    const Species& S = c.sp[s];
    if (S.n > 0) k_set_temperature<<<grid_of(c, S.n), 256, 0, st>>>(S.a.cell, S.a.ux, S.a.uy, S.a.uz, S.n, T, T_from);
}

}  // namespace gbpic
