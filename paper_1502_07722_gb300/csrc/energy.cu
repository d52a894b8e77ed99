// Energy diagnostics in FP64 (paper: the pair-potential cycle is energy conserving):
// kinetic energy per species, electric and magnetic field energy, pair-potential energy.
// Each block reduces its share into a fixed slot of a partials array; a single block then adds
// the partials in block order, so the result does not depend on scheduling.
#include "pic_device.cuh"

namespace gbpic {

constexpr int kEBlock = 256;
constexpr int kSlots = 5;   // 0 KE ions, 1 KE electrons, 2 field E, 3 field B, 4 pair

__device__ __forceinline__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kEBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

struct EnergyArgs {
    int nx, nz, nsp;
    SpeciesBuf sp[2];
    int64_t n[2];
    const float* F[6];
    const u64* rho;
    float rho_s, h_coef, c_att, s_rep;
    int pot_mode;
    EamP eam;
    double* partials;   // gridDim.x * kSlots
};

__global__ void __launch_bounds__(kEBlock) k_energy(const EnergyArgs a)
{
    __shared__ double sh[kEBlock];
    const int64_t tid = blockIdx.x * (int64_t)kEBlock + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kEBlock;
    double ke[2] = {0.0, 0.0}, pe = 0.0, fe = 0.0, fb = 0.0;
#pragma unroll
    for (int s = 0; s < 2; s++) {
        if (s >= a.nsp) break;
        const SpeciesBuf& S = a.sp[s];
        for (int64_t p = tid; p < a.n[s]; p += stride) {
            const float ux = S.ux[p], uy = S.uy[p], uz = S.uz[p];
            const float u2 = ux * ux + uy * uy + uz * uz;
            ke[s] += (double)(u2 / (sqrtf(1.0f + u2) + 1.0f));
            if (s == 0) {
                const int c = S.cell[p];
                const int k = c / a.nx, i = c - k * a.nx;
                float n, dnx, dnz;
                gather_density(a.rho, a.nx, a.nz, a.rho_s, i, k, S.fx[p], S.fz[p], n, dnx, dnz);
                if (n > 0.0f) {
                    const float cr = fast_cbrt(n);
                    const float inv43 = fast_rcp(n * cr);
                    float e = pair_energy_xz(cr, inv43, dnx, dnz, a.h_coef, a.pot_mode, a.c_att, a.s_rep, a.eam);
                    pe += (double)e;
                }
            }
        }
    }
    const int64_t nn = (int64_t)(a.nz + 1) * a.nx;
    for (int64_t c = tid; c < nn; c += stride) {
        const int k = (int)(c / a.nx);
        const double wn = (k == 0 || k == a.nz) ? 0.5 : 1.0;
        const double ex = a.F[0][c], ey = a.F[1][c], bz = a.F[5][c];
        fe += wn * (ex * ex + ey * ey);
        fb += wn * bz * bz;
        if (k < a.nz) {
            const double ez = a.F[2][c], bx = a.F[3][c], by = a.F[4][c];
            fe += ez * ez;
            fb += bx * bx + by * by;
        }
    }
    const double r0 = block_sum(ke[0], sh), r1 = block_sum(ke[1], sh), r2 = block_sum(fe, sh),
                 r3 = block_sum(fb, sh), r4 = block_sum(pe, sh);
    if (threadIdx.x == 0) {
        double* o = a.partials + (size_t)blockIdx.x * kSlots;
        o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3; o[4] = r4;
    }
}

__global__ void k_energy_final(const double* __restrict__ partials, int nb, double* out)
{
    __shared__ double sh[kEBlock];
    for (int s = 0; s < kSlots; s++) {
        double v = 0.0;
        // fixed assignment of blocks to threads, then a fixed-shape tree
        for (int b = threadIdx.x; b < nb; b += kEBlock) v += partials[(size_t)b * kSlots + s];
        const double r = block_sum(v, sh);
        if (threadIdx.x == 0) out[s] = r;
    }
}

int energy_blocks(const Ctx& c) { return c.nsm * 4; }

void launch_energy(Ctx& c, cudaStream_t st, double* host_out5)
{
    EnergyArgs a;
    a.nx = c.nx;
    a.nz = c.nz;
    a.nsp = c.nsp;
    for (int s = 0; s < 2; s++) {
        a.sp[s] = c.sp[s].a;
        a.n[s] = c.sp[s].n;
    }
    for (int q = 0; q < 6; q++) a.F[q] = c.F[q];
    a.rho = c.rho[c.cur];
    a.rho_s = (float)c.rho_scale;
    a.h_coef = (float)(c.r0 / (6.0 * c.cfg.dx));
    a.c_att = pot_param(c.cfg);
    a.s_rep = (float)c.cfg.s_rep;
    a.pot_mode = pot_code(c.cfg);
    a.eam = eam_params(c.cfg);
    a.partials = c.partials;
    const int nb = energy_blocks(c);
    k_energy<<<nb, kEBlock, 0, st>>>(a);
    k_energy_final<<<1, kEBlock, 0, st>>>(c.partials, nb, c.red_out);
    double raw[kSlots];
    cudaMemcpyAsync(raw, c.red_out, sizeof(raw), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    const double vol = c.cfg.dx * c.cfg.dx;
    const double mu0 = 1.0 / (kEps0 * kC * kC);
    host_out5[0] = raw[0] * c.w * c.sp[0].mass * kC * kC;
    host_out5[1] = c.nsp > 1 ? raw[1] * c.w * c.sp[1].mass * kC * kC : 0.0;
    host_out5[2] = 0.5 * kEps0 * raw[2] * vol;
    host_out5[3] = 0.5 / mu0 * raw[3] * vol;
    host_out5[4] = 0.5 * c.D * raw[4] * c.w;
}

}  // namespace gbpic

// ---------------------------------------------------------------------------------------------
// Workspace-free variant of the energy reduction (pic_energy_noalloc in include/pic.h).
//
// Some callers cannot allocate device memory at all: a host that hands this library buffers it
// owns but forbids further cudaMalloc (a caller-managed memory pool, or code that must not
// allocate while a CUDA graph is being recorded by someone else). For them the reduction's
// scratch -- one partial-sum record per block -- lives in a fixed array in this translation unit,
// reserved on every GPU that loads the library until the process exits.
// ---------------------------------------------------------------------------------------------

namespace gbpic {

constexpr int kStaticBlocks = 1024;                     // partial records the fixed scratch holds
static __device__ __align__(256) double g_noalloc_scratch[kStaticBlocks * kSlots];

// Final pass of the workspace-free variant: adds the block partials in block order (the same
// fixed-shape tree as k_energy_final) and writes the five energies in J per metre of y.
__global__ void k_energy_final_scaled(const double* __restrict__ partials, int nb, double s0, double s1, double s2,
                                      double s3, double s4, double* out)
{
    __shared__ double sh[kEBlock];
    const double scale[kSlots] = {s0, s1, s2, s3, s4};
    for (int s = 0; s < kSlots; s++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += kEBlock) v += partials[(size_t)b * kSlots + s];
        const double r = block_sum(v, sh);
        if (threadIdx.x == 0) out[s] = r * scale[s];
    }
}

}  // namespace gbpic

#include <mutex>

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the fixed scratch on the current device. The symbol name is only a host-side
// handle: its device address comes from cudaGetSymbolAddress, taken once per device with that
// device current, on the first call.
int noalloc_scratch(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, gbpic::g_noalloc_scratch) != cudaSuccess || !p) return PIC_ECUDA;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return PIC_OK;
}

}  // namespace

extern "C" int pic_energy_noalloc(const pic_config* cfg, const pic_state_view* in, double* dev_out5, void* stream)
{
    using namespace gbpic;
    if (!cfg || !in || !dev_out5) return PIC_EINVAL;
    if (cfg->dims != 0 && cfg->dims != 2) return PIC_EINVAL;     // 2D states only
    if (cfg->nx < 3 || cfg->nz < 4 || cfg->nx >= 32768 || cfg->nz >= 32768) return PIC_EINVAL;
    if (cfg->mode != PIC_MODE_FULL && cfg->mode != PIC_MODE_TRANSPORT) return PIC_EINVAL;
    if (!(cfg->dx > 0) || !(cfg->n_atoms > 0) || !(cfg->ion_mass_amu > 0) || cfg->ppc_ion <= 0) return PIC_EINVAL;
    if (cfg->pot_mode < 0 || cfg->pot_mode > 3) return PIC_EINVAL;
    if (cfg->pot_mode == 2 && !(cfg->morse_a > 0 && cfg->morse_a < 1e3)) return PIC_EINVAL;
    if (cfg->lattice != PIC_LATTICE_CUBIC && cfg->lattice != PIC_LATTICE_HCP) return PIC_EINVAL;
    if (!eam_config_ok(*cfg)) return PIC_EINVAL;
    const int nsp = cfg->mode == PIC_MODE_FULL ? 2 : 1;
    for (int s = 0; s < nsp; s++) {
        // sizes beyond what the kernels index with 32-bit cells are refused
        if (in->n[s] < 0 || in->n[s] > (int64_t)INT32_MAX) return PIC_EINVAL;
        if (in->n[s] > 0 && (!in->cell[s] || !in->fx[s] || !in->fz[s] || !in->ux[s] || !in->uy[s] || !in->uz[s]))
            return PIC_EINVAL;
    }
    for (int q = 0; q < 6; q++)
        if (!in->F[q]) return PIC_EINVAL;
    if (!in->rho) return PIC_EINVAL;

    double* scratch = nullptr;
    int r = noalloc_scratch(&scratch);
    if (r) return r;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIC_ECUDA;
    const int nb = nsm * 4 < kStaticBlocks ? nsm * 4 : kStaticBlocks;

    // derived constants, as pic_init derives them
    const double w = cfg->n_atoms * cfg->dx * cfg->dx / (double)cfg->ppc_ion;
    const double r0 = cfg->r0 > 0 ? cfg->r0 : pow(cfg->n_atoms, -1.0 / 3.0);
    const double D = cfg->D_eV * kQe;
    const double rho_scale = w / (4294967296.0 * cfg->dx * cfg->dx) * r0 * r0 * r0;
    const double mi = cfg->ion_mass_amu * kAmu;

    EnergyArgs a;
    a.nx = cfg->nx;
    a.nz = cfg->nz;
    a.nsp = nsp;
    for (int s = 0; s < 2; s++) {
        const bool on = s < nsp;
        a.sp[s].cell = on ? const_cast<int32_t*>(in->cell[s]) : nullptr;
        a.sp[s].fx = on ? const_cast<float*>(in->fx[s]) : nullptr;
        a.sp[s].fz = on ? const_cast<float*>(in->fz[s]) : nullptr;
        a.sp[s].ux = on ? const_cast<float*>(in->ux[s]) : nullptr;
        a.sp[s].uy = on ? const_cast<float*>(in->uy[s]) : nullptr;
        a.sp[s].uz = on ? const_cast<float*>(in->uz[s]) : nullptr;
        a.n[s] = on ? in->n[s] : 0;
    }
    for (int q = 0; q < 6; q++) a.F[q] = in->F[q];
    a.rho = reinterpret_cast<const u64*>(in->rho);
    a.rho_s = (float)rho_scale;
    a.h_coef = (float)(r0 / (6.0 * cfg->dx));
    a.c_att = pot_param(*cfg);
    a.s_rep = (float)cfg->s_rep;
    a.pot_mode = pot_code(*cfg);
    a.eam = eam_params(*cfg);
    a.partials = scratch;    // every block overwrites its own record: nothing to clear
    const cudaStream_t st = (cudaStream_t)stream;
    const double vol = cfg->dx * cfg->dx;
    const double mu0 = 1.0 / (kEps0 * kC * kC);
    k_energy<<<nb, kEBlock, 0, st>>>(a);
    k_energy_final_scaled<<<1, kEBlock, 0, st>>>(scratch, nb, w * mi * kC * kC, nsp > 1 ? w * kMe * kC * kC : 0.0,
                                                  0.5 * kEps0 * vol, 0.5 / mu0 * vol, 0.5 * D * w, dev_out5);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
