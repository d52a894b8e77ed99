// Crater profile of the atomic-transport stage (paper: once the crater has solidified its width
// and depth are measured from the density map and compared with experiment; Eq. 5 turns the
// width into a threshold fluence). For every column of nodes the material missing from the
// original slab, as a thickness of solid-density material:
//     d(column) = dx * scale / n_atoms * sum_{k = 0..slab_k} (rho0 - rho)(k, column),
// rho0 the node sums at the start, rho the current ones (int64 node sums of the pair species),
// scale the factor from a node sum to a density in m^-3. The column sums are exact integers; one
// FP64 multiply per column turns them into metres.
#include "pic_internal.cuh"

namespace gbpic {

__global__ void k_crater_profile(const u64* __restrict__ rho0, const u64* __restrict__ rho, int64_t ncol,
                                 int rows, double depth_scale, double* __restrict__ out)
{
    for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < ncol;
         col += (int64_t)gridDim.x * blockDim.x) {
        long long s = 0;
        for (int k = 0; k < rows; k++) {
            const size_t q = (size_t)k * (size_t)ncol + (size_t)col;
            s += (long long)(__ldg(rho0 + q) - __ldg(rho + q));
        }
        out[col] = (double)s * depth_scale;
    }
}

void launch_crater_profile(Ctx& c, const u64* rho0, double depth_scale, double* out, cudaStream_t st)
{
    const int64_t ncol = (int64_t)c.nx * c.ny;
    const int rows = c.cfg.slab_k + 1 < c.nz + 1 ? c.cfg.slab_k + 1 : c.nz + 1;
    int64_t g = (ncol + 255) / 256;
    if (g > (int64_t)c.nsm * 8) g = (int64_t)c.nsm * 8;
    k_crater_profile<<<(int)g, 256, 0, st>>>(rho0, c.rho[c.cur], ncol, rows, depth_scale, out);
}

}  // namespace gbpic
