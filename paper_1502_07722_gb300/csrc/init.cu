// Initial state of a damage simulation (paper: the simulation is initialised for target density
// and temperature): ppc macroparticles per slab cell at uniformly drawn offsets, Maxwellian
// momenta at a uniform temperature or, for species 0, at the local lattice temperature of a laser
// spot; electrons reuse the ion positions so the start is neutral with E = 0.
//
// Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used counter-style, one draw =
// the first output of a generator seeded with seed ^ key, key = ((species 2^40 + particle) 8 + d).
// Uniform offsets take the top 24 bits (exact in FP32); normals come from Box-Muller in FP64.
#include "pic_internal.cuh"

namespace gbpic {

__device__ __forceinline__ uint64_t smix_first(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t seed, int s, uint64_t pid, int d)
{
    return smix_first(seed ^ (((((uint64_t)s << 40) + pid) << 3) + (uint64_t)d));
}

// Lattice temperature of a laser spot (PIC_TEMP_SPOT): T at the particle's initial position in
// cells, Gaussian in the lateral distance from the spot axis (x in 2D, the radius in the x-y plane
// in 3D) and exponential in the depth below the slab surface; the thermal momentum scale is
// sqrt(k_B T / (m c^2)) with the same operation order as the uniform case.
struct TempSpot {
    int on;
    double T_base, T_spot;     // K
    double xc, yc, zs;         // axis (cells) and slab surface row
    double cx, cz;             // dx / spot_w, dx / spot_depth
    double kb, mc2;            // k_B, m c^2
};

__device__ __forceinline__ double spot_uth(const TempSpot& ts, double ex2, double z)
{
    const double T = ts.T_base + (ts.T_spot - ts.T_base) * exp(-2.0 * ex2) * exp(-(ts.zs - z) * ts.cz);
    return sqrt(ts.kb * T / ts.mc2);
}

static TempSpot temp_spot(const Ctx& c, int s)
{
    TempSpot ts = {};
    if (s == 0 && c.cfg.temp_profile == PIC_TEMP_SPOT) {
        ts.on = 1;
        ts.T_base = c.cfg.T_ion_K;
        ts.T_spot = c.cfg.T_spot_K;
        ts.xc = 0.5 * c.nx;
        ts.yc = 0.5 * c.ny;
        ts.zs = c.cfg.slab_k;
        ts.cx = c.cfg.dx / c.cfg.spot_w;
        ts.cz = c.cfg.dx / c.cfg.spot_depth;
        ts.kb = kKb;
        ts.mc2 = c.sp[s].mass * kC * kC;
    }
    return ts;
}

__global__ void k_init(SpeciesBuf out, int64_t n, int ppc, int nx, int species, int pos_species, double uth,
                       uint64_t seed, TempSpot ts)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t cellidx = (uint64_t)p / (uint64_t)ppc;     // row-major slab cell
        const int k = (int)(cellidx / (uint64_t)nx);
        const int i = (int)(cellidx - (uint64_t)k * nx);
        out.cell[p] = k * nx + i;
        out.fx[p] = (float)(draw(seed, pos_species, (uint64_t)p, 0) >> 40) * (1.0f / 16777216.0f);
        out.fz[p] = (float)(draw(seed, pos_species, (uint64_t)p, 1) >> 40) * (1.0f / 16777216.0f);
        const double u1 = ((double)(draw(seed, species, (uint64_t)p, 2) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double a1 = 2.0 * kPi * (double)(draw(seed, species, (uint64_t)p, 3) >> 40) * (1.0 / 16777216.0);
        const double u2 = ((double)(draw(seed, species, (uint64_t)p, 4) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double a2 = 2.0 * kPi * (double)(draw(seed, species, (uint64_t)p, 5) >> 40) * (1.0 / 16777216.0);
        const double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u2));
        double u = uth;
        if (ts.on) {
            const double x = (double)i + (double)out.fx[p], z = (double)k + (double)out.fz[p];
            const double ex = (x - ts.xc) * ts.cx;
            u = spot_uth(ts, ex * ex, z);
        }
        out.ux[p] = (float)(u * r1 * cos(a1));
        out.uy[p] = (float)(u * r1 * sin(a1));
        out.uz[p] = (float)(u * r2 * cos(a2));
    }
}

void launch_init_particles(Ctx& c, int s, cudaStream_t st)
{
    Species& S = c.sp[s];
    if (S.n == 0) return;
    int64_t g = (S.n + 255) / 256;
    if (g > (int64_t)c.nsm * 16) g = (int64_t)c.nsm * 16;
    const int pos_species = (s == 1 && c.cfg.ppc_electron == c.cfg.ppc_ion) ? 0 : s;
    const TempSpot ts = temp_spot(c, s);
    k_init<<<(int)g, 256, 0, st>>>(S.b, S.n, S.ppc, c.nx, s, pos_species, S.uth, c.cfg.seed, ts);
}

// 3D: slab cells k < slab_k over all (i, j), row-major; positions from draws 0 (x), 6 (y), 1 (z)
__global__ void k_init3(SpeciesBuf out, int64_t n, int ppc, int nx, int ny, int species, int pos_species, double uth,
                        uint64_t seed, TempSpot ts)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t cellidx = (uint64_t)p / (uint64_t)ppc;
        out.cell[p] = (int32_t)cellidx;
        out.fx[p] = (float)(draw(seed, pos_species, (uint64_t)p, 0) >> 40) * (1.0f / 16777216.0f);
        out.fy[p] = (float)(draw(seed, pos_species, (uint64_t)p, 6) >> 40) * (1.0f / 16777216.0f);
        out.fz[p] = (float)(draw(seed, pos_species, (uint64_t)p, 1) >> 40) * (1.0f / 16777216.0f);
        const double u1 = ((double)(draw(seed, species, (uint64_t)p, 2) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double a1 = 2.0 * kPi * (double)(draw(seed, species, (uint64_t)p, 3) >> 40) * (1.0 / 16777216.0);
        const double u2 = ((double)(draw(seed, species, (uint64_t)p, 4) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double a2 = 2.0 * kPi * (double)(draw(seed, species, (uint64_t)p, 5) >> 40) * (1.0 / 16777216.0);
        const double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u2));
        double u = uth;
        if (ts.on) {
            const uint64_t row = cellidx / (uint64_t)nx;
            const int i = (int)(cellidx - row * (uint64_t)nx);
            const int k = (int)(row / (uint64_t)ny);
            const int j = (int)(row - (uint64_t)k * ny);
            const double x = (double)i + (double)out.fx[p], y = (double)j + (double)out.fy[p];
            const double z = (double)k + (double)out.fz[p];
            const double ex = (x - ts.xc) * ts.cx, ey = (y - ts.yc) * ts.cx;
            u = spot_uth(ts, ex * ex + ey * ey, z);
        }
        out.ux[p] = (float)(u * r1 * cos(a1));
        out.uy[p] = (float)(u * r1 * sin(a1));
        out.uz[p] = (float)(u * r2 * cos(a2));
    }
}

void launch_init_particles3(Ctx& c, int s, cudaStream_t st)
{
    Species& S = c.sp[s];
    if (S.n == 0) return;
    int64_t g = (S.n + 255) / 256;
    if (g > (int64_t)c.nsm * 16) g = (int64_t)c.nsm * 16;
    const int pos_species = (s == 1 && c.cfg.ppc_electron == c.cfg.ppc_ion) ? 0 : s;
    k_init3<<<(int)g, 256, 0, st>>>(S.b, S.n, S.ppc, c.nx, c.ny, s, pos_species, S.uth, c.cfg.seed,
                                    temp_spot(c, s));
}

}  // namespace gbpic
