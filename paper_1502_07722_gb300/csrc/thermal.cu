// Coupling of the two stages (paper: the atomic-transport run starts from the lattice temperature
// the laser-interaction run leaves once electrons and lattice have equilibrated).
//  * Lattice temperature per cell of one species: T = m c^2 / (3 k_B) sum |u - mean u|^2 / (N - 1)
//    over the N particles of the cell (the thermal spread about the cell's mean flow); cells with
//    fewer than two particles get 0. Per-cell sums in FP64 (atomics), then one thread per cell.
//  * Re-tempering to a map: momenta drawn at the uniform temperature T_from become the same draws
//    at the temperature of their cell, u -> u sqrt(T_cell / T_from).
//  * Regridding a cell map between stages of different cells: a conservative (volume-weighted)
//    remap on grids placed on each other by the slab's surface and the laser axis.
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

// One axis of the remap: destination cell d of a grid (n, dx, origin o: cell d spans
// [(d - o) dx, (d + 1 - o) dx]) against the source axis (ns, dxs, os); the source cells it overlaps
// are lo .. hi (empty when lo > hi), the overlap with source cell s is ov(s).
struct RegridAxis {
    double a0, a1, dxs, os;
    int lo, hi;
};
__device__ __forceinline__ RegridAxis regrid_axis(int d, double dx, double o, int ns, double dxs, double os)
{
    RegridAxis A;
    A.a0 = (d - o) * dx;
    A.a1 = (d + 1 - o) * dx;
    A.dxs = dxs;
    A.os = os;
    A.lo = max(0, (int)floor(A.a0 / dxs + os));
    A.hi = min(ns - 1, (int)ceil(A.a1 / dxs + os) - 1);
    return A;
}
__device__ __forceinline__ double regrid_overlap(const RegridAxis& A, int s)
{
    const double b0 = (s - A.os) * A.dxs, b1 = b0 + A.dxs;
    return fmax(0.0, fmin(A.a1, b1) - fmax(A.a0, b0));
}

struct RegridGrid {
    int nx, ny, nz;
    double dx, ox, oy, oz;      // origins: nx / 2, ny / 2, surface
};

__global__ void k_regrid_cells(int dims, const double* __restrict__ src, RegridGrid S, double* __restrict__ dst,
                               RegridGrid D, double fill)
{
    const int64_t nd = (int64_t)D.nx * D.ny * D.nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nd; c += stride) {
        const int i = (int)(c % D.nx);
        const int64_t q = c / D.nx;
        const int j = (int)(q % D.ny), k = (int)(q / D.ny);
        const RegridAxis X = regrid_axis(i, D.dx, D.ox, S.nx, S.dx, S.ox);
        const RegridAxis Z = regrid_axis(k, D.dx, D.oz, S.nz, S.dx, S.oz);
        RegridAxis Y;
        if (dims == 3) Y = regrid_axis(j, D.dx, D.oy, S.ny, S.dx, S.oy);
        double sum = 0.0, covered = 0.0;
        for (int sk = Z.lo; sk <= Z.hi; sk++) {
            const double wz = regrid_overlap(Z, sk);
            for (int sj = dims == 3 ? Y.lo : 0; sj <= (dims == 3 ? Y.hi : 0); sj++) {
                const double wzy = dims == 3 ? wz * regrid_overlap(Y, sj) : wz;
                for (int si = X.lo; si <= X.hi; si++) {
                    const double w = wzy * regrid_overlap(X, si);
                    sum += w * src[((int64_t)sk * S.ny + sj) * S.nx + si];
                    covered += w;
                }
            }
        }
        const double vol = dims == 3 ? D.dx * D.dx * D.dx : D.dx * D.dx;
        dst[c] = (sum + fill * (vol - covered)) / vol;
    }
}

}  // namespace gbpic

extern "C" PIC_API int pic_regrid_cells(int32_t dims, const double* dev_src, int32_t src_nx, int32_t src_ny,
                                        int32_t src_nz, double src_dx, int32_t src_surface, double* dev_dst,
                                        int32_t dst_nx, int32_t dst_ny, int32_t dst_nz, double dst_dx,
                                        int32_t dst_surface, double fill, void* stream)
{
    using namespace gbpic;
    if (!dev_src || !dev_dst || (dims != 2 && dims != 3)) return PIC_EINVAL;
    if (dims == 2) src_ny = dst_ny = 1;
    if (src_nx < 1 || src_ny < 1 || src_nz < 1 || dst_nx < 1 || dst_ny < 1 || dst_nz < 1) return PIC_EINVAL;
    if (!(src_dx > 0.0) || !(dst_dx > 0.0)) return PIC_EINVAL;
    if (src_surface < 0 || src_surface > src_nz || dst_surface < 0 || dst_surface > dst_nz) return PIC_EINVAL;
    const RegridGrid S = {src_nx, src_ny, src_nz, src_dx, 0.5 * src_nx, 0.5 * src_ny, (double)src_surface};
    const RegridGrid D = {dst_nx, dst_ny, dst_nz, dst_dx, 0.5 * dst_nx, 0.5 * dst_ny, (double)dst_surface};
    const int64_t nd = (int64_t)dst_nx * dst_ny * dst_nz;
    int64_t g = (nd + 255) / 256;
    if (g > 65536) g = 65536;
    k_regrid_cells<<<(int)g, 256, 0, (cudaStream_t)stream>>>(dims, dev_src, S, dev_dst, D, fill);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

