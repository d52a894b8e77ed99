// Host side of the C ABI declared in include/pic.h: configuration, workspace layout, the step
// loop and data movement. Every operation of the cycle itself runs in the kernels of this
// directory; nothing here computes on particles or grids.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pic_internal.cuh"

namespace gbpic {
int tile_window(int T);
int energy_blocks(const Ctx& c);
void sort_species_impl(Ctx& c, int s, cudaStream_t st, int from_b, int64_t* launches);
}  // namespace gbpic

using namespace gbpic;

#define CK(x)                                              \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) return PIC_ECUDA;           \
    } while (0)

namespace {

constexpr int kMaxEnergyBlocks = 1024;

struct Layout {
    int32_t dims, nx, ny, nz, T, ntx, nty, ntz, ntiles, nkeys, nsp, jy_bits;
    int64_t count_limit;
    size_t nn;
    int64_t cap[2], n0[2];
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int derive_layout(const pic_config* cfg, Layout& L)
{
    if (!cfg) return PIC_EINVAL;
    L.dims = cfg->dims == 0 ? 2 : cfg->dims;
    if (L.dims != 2 && L.dims != 3) return PIC_EINVAL;
    L.ny = L.dims == 3 ? cfg->ny : 1;
    if (cfg->nx < 3 || cfg->nz < 4 || cfg->nx >= 32768 || cfg->nz >= 32768) return PIC_EINVAL;
    if (L.dims == 3 && (L.ny < 3 || L.ny >= 32768 || (int64_t)cfg->nx * L.ny * (cfg->nz + 1) >= (1LL << 31)))
        return PIC_EINVAL;
    if (cfg->slab_k < 0 || cfg->slab_k > cfg->nz) return PIC_EINVAL;
    if (cfg->mode != PIC_MODE_FULL && cfg->mode != PIC_MODE_TRANSPORT) return PIC_EINVAL;
    if (cfg->ppc_ion < 0 || cfg->ppc_electron < 0) return PIC_EINVAL;
    if (!(cfg->dx > 0) || !(cfg->n_atoms > 0) || !(cfg->ion_mass_amu > 0)) return PIC_EINVAL;
    if (cfg->dt_override <= 0 && !(cfg->cfl > 0 && cfg->cfl <= 1.0)) return PIC_EINVAL;
    if (cfg->mode == PIC_MODE_FULL) {
        if (cfg->ion_charge != 1.0) return PIC_EINVAL;            // equal |q| w across species
        if (cfg->ppc_electron != cfg->ppc_ion) return PIC_EINVAL;
    } else if (cfg->ion_charge != 0.0) {
        return PIC_EINVAL;
    }
    if (cfg->laser_profile < 0 || cfg->laser_profile > 2) return PIC_EINVAL;
    if (cfg->laser_profile != PIC_LASER_NONE && cfg->mode == PIC_MODE_FULL &&
        !(cfg->lambda > 0 && cfg->tau_fwhm > 0))
        return PIC_EINVAL;
    if (cfg->laser_profile == PIC_LASER_GAUSSIAN && !(cfg->w0 > 0)) return PIC_EINVAL;
    if (cfg->pot_mode < 0 || cfg->pot_mode > 3) return PIC_EINVAL;
    if (cfg->pot_mode == 2 && !(cfg->morse_a > 0 && cfg->morse_a < 1e3)) return PIC_EINVAL;
    if (cfg->lattice != PIC_LATTICE_CUBIC && cfg->lattice != PIC_LATTICE_HCP) return PIC_EINVAL;
    if (!eam_config_ok(*cfg)) return PIC_EINVAL;
    if (cfg->temp_profile != PIC_TEMP_UNIFORM && cfg->temp_profile != PIC_TEMP_SPOT) return PIC_EINVAL;
    if (cfg->temp_profile == PIC_TEMP_SPOT &&
        (!(cfg->spot_w > 0) || !(cfg->spot_depth > 0) || !(cfg->T_spot_K >= 0)))
        return PIC_EINVAL;
    L.nx = cfg->nx;
    L.nz = cfg->nz;
    L.T = cfg->tile > 0 ? cfg->tile : (L.dims == 3 ? 10 : 16);
    if (L.T < 2 || L.T > 64) return PIC_EINVAL;
    L.ntx = (L.nx + L.T - 1) / L.T;
    L.nty = L.dims == 3 ? (L.ny + L.T - 1) / L.T : 1;
    L.ntz = (L.nz + L.T - 1) / L.T;
    L.ntiles = L.ntx * L.nty * L.ntz;
    const int64_t nkeys = (int64_t)L.ntiles * L.T * L.T * (L.dims == 3 ? L.T : 1);
    if (nkeys >= (1LL << 31) - 1) return PIC_EINVAL;
    L.nkeys = (int32_t)nkeys;
    L.nn = (size_t)L.nx * L.ny * (L.nz + 1);
    L.nsp = cfg->mode == PIC_MODE_FULL ? 2 : 1;
    const int64_t ncell = (int64_t)cfg->nx * L.ny * cfg->slab_k;
    for (int s = 0; s < 2; s++) {
        const int ppc = s == 0 ? cfg->ppc_ion : cfg->ppc_electron;
        L.n0[s] = s < L.nsp ? ncell * ppc : 0;
        L.cap[s] = s < L.nsp ? (cfg->max_particles > 0 ? cfg->max_particles : L.n0[s]) : 0;
        if (L.cap[s] < L.n0[s] || L.cap[s] >= (1LL << 31)) return PIC_EINVAL;
    }
    // fixed-point range of the node sums (PIC_EOVERFLOW): the initial particles per cell must fit
    const int64_t per_cell = (int64_t)(cfg->ppc_ion > 0 ? cfg->ppc_ion : 0) + (L.nsp > 1 ? cfg->ppc_electron : 0);
    const int full = cfg->mode == PIC_MODE_FULL;
    L.jy_bits = (L.dims == 2 && full) ? choose_jy_bits(per_cell) : 18;
    if (L.jy_bits < 1) return PIC_EOVERFLOW;
    L.count_limit = count_limit(L.dims, full, L.jy_bits);
    if ((L.dims == 3 ? 64 : 16) * per_cell > L.count_limit) return PIC_EOVERFLOW;
    size_t t = 0;
    const int arrays = L.dims == 3 ? 7 : 6;
    for (int s = 0; s < 2; s++) t += 2 * arrays * align256(4 * (size_t)L.cap[s]) + align256(4 * (size_t)(L.ntiles + 1));
    t += 6 * align256(4 * L.nn) + 5 * align256(8 * L.nn);
    const size_t plane = (size_t)L.nx * L.ny;
    t += align256(4 * 8 * plane) + 2 * align256(4 * plane) + align256(8);
    t += 2 * align256(4 * ((size_t)L.nkeys + 1));
    t += align256(4 * (((size_t)L.nkeys + 2047) / 2048 + 1));
    t += align256(8 * 5 * (size_t)kMaxEnergyBlocks) + align256(8 * 8) + align256(32);
    L.total = t;
    return PIC_OK;
}

struct Carver {
    char* p;
    char* end;
    template <class T>
    T* take(size_t count)
    {
        T* r = reinterpret_cast<T*>(p);
        p += align256(sizeof(T) * count);
        return r;
    }
};

int finish_status(pic_ctx* h)
{
    Ctx& c = h->c;
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, c.status, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (c.timing) {
        for (size_t j = 0; j + 1 < h->evpool.size() && j / 2 < h->evkind.size(); j += 2) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->evpool[j], h->evpool[j + 1]));
            const int kind = h->evkind[j / 2];
            c.ms[kind] += ms;
        }
        h->evkind.clear();
    }
    if (st & kErrNan) c.sticky = PIC_ENAN;
    else if (st & kErrMove) c.sticky = PIC_EMOVE;
    else if (st & kErrOverflow) c.sticky = PIC_EOVERFLOW;
    return c.sticky;
}

int ev_begin(pic_ctx* h, int kind)
{
    if (!h->c.timing) return PIC_OK;
    const size_t j = 2 * h->evkind.size();
    while (h->evpool.size() < j + 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->evpool.push_back(e);
    }
    h->evkind.push_back(kind);
    CK(cudaEventRecord(h->evpool[j], h->c.stream));
    return PIC_OK;
}

int ev_end(pic_ctx* h)
{
    if (!h->c.timing) return PIC_OK;
    const size_t j = 2 * h->evkind.size() - 1;
    CK(cudaEventRecord(h->evpool[j], h->c.stream));
    return PIC_OK;
}

int sort_all(pic_ctx* h)
{
    Ctx& c = h->c;
    int r = ev_begin(h, 2);
    if (r) return r;
    const int64_t before = c.nlaunch[2];
    for (int s = 0; s < c.nsp; s++) launch_sort_species(c, s, c.stream, &c.nlaunch[2]);
    c.nlaunch[3] += c.nlaunch[2] - before;
    r = ev_end(h);
    if (r) return r;
    CK(cudaGetLastError());
    c.steps_since_sort = 0;
    return PIC_OK;
}

int redeposit(Ctx& c)
{
    if (c.dims == 3) launch_deposit_density3(c, c.rho[c.cur], c.stream);
    else launch_deposit_density(c, c.rho[c.cur], c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

}  // namespace

namespace gbpic {

StepArgs make_step_args(Ctx& c)
{
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = c.nx;
    a.nz = c.nz;
    a.T = c.T;
    a.ntx = c.ntx;
    a.ntz = c.ntz;
    a.ntiles = c.ntiles;
    a.W = c.W;
    a.nx_magic = (unsigned)(4294967296ULL / (unsigned long long)c.nx);
    a.full = c.cfg.mode == PIC_MODE_FULL;
    a.cdt_dx = (float)(kC * c.dt / c.cfg.dx);
    a.rho_s = (float)c.rho_scale;
    a.h_coef = (float)(c.r0 / (6.0 * c.cfg.dx));
    a.pot_mode = pot_code(c.cfg);
    a.c_att = pot_param(c.cfg);
    a.s_rep = (float)c.cfg.s_rep;
    for (int q = 0; q < 6; q++) a.F[q] = c.F[q];
    a.rho_cur = c.rho[c.cur];
    a.rho_next = c.rho[1 - c.cur];
    for (int q = 0; q < 3; q++) a.J[q] = c.J[q];
    a.status = c.status;
    a.nsp = c.nsp;
    for (int s = 0; s < 2; s++) a.sp[s] = c.sp[s];
    a.eam = eam_params(c.cfg);
    a.jy_scale = ldexpf(1.0f, c.jy_bits);
    a.jy_zero = ldexpf(1.0f, -(c.jy_bits + 1));
    return a;
}

}  // namespace gbpic

extern "C" {

size_t pic_config_bytes(void) { return sizeof(pic_config); }

int pic_workspace_size(const pic_config* cfg, size_t* bytes)
{
    if (!bytes) return PIC_EINVAL;
    Layout L;
    int r = derive_layout(cfg, L);
    if (r) return r;
    *bytes = L.total;
    return PIC_OK;
}

int pic_init(const pic_config* cfg, void* workspace, size_t workspace_bytes, void* stream, pic_ctx** out)
{
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    Layout L;
    int r = derive_layout(cfg, L);
    if (r) return r;
    if (!workspace || ((uintptr_t)workspace & 255)) return PIC_EINVAL;
    if (workspace_bytes < L.total) return PIC_ENOMEM;
    pic_ctx* h = new (std::nothrow) pic_ctx();
    if (!h) return PIC_ENOMEM;
    Ctx& c = h->c;
    c.cfg = *cfg;
    c.stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) {
        delete h;
        return PIC_ECUDA;
    }
    c.dims = L.dims;
    c.nx = L.nx;
    c.ny = L.ny;
    c.nz = L.nz;
    c.T = L.T;
    c.ntx = L.ntx;
    c.nty = L.nty;
    c.ntz = L.ntz;
    c.ntiles = L.ntiles;
    c.W = tile_window(L.T);
    c.nkeys = L.nkeys;
    c.nn = L.nn;
    c.nsp = L.nsp;
    c.k_ant = L.nz - 2;
    c.jy_bits = L.jy_bits;
    c.count_limit = (int32_t)(L.count_limit < 2147483647 ? L.count_limit : 2147483647);
    // derived physics
    const bool d3 = L.dims == 3;
    c.dt = cfg->dt_override > 0 ? cfg->dt_override : cfg->cfl * cfg->dx / (kC * sqrt(d3 ? 3.0 : 2.0));
    // atoms per macroparticle (per metre of y in 2D)
    c.w = cfg->n_atoms * cfg->dx * cfg->dx * (d3 ? cfg->dx : 1.0) / (double)(cfg->ppc_ion > 0 ? cfg->ppc_ion : 1);
    c.r0 = cfg->r0 > 0 ? cfg->r0 : pow(cfg->n_atoms, -1.0 / 3.0);
    c.D = cfg->D_eV * kQe;
    // node sum -> n / n0; a node sum counts one macroparticle as 2^32 (2D) or 2^42 (3D)
    c.rho_scale = d3 ? c.w / (4398046511104.0 * cfg->dx * cfg->dx * cfg->dx) * c.r0 * c.r0 * c.r0
                     : c.w / (4294967296.0 * cfg->dx * cfg->dx) * c.r0 * c.r0 * c.r0;
    c.E0 = sqrt(2.0 * cfg->I0 / (kEps0 * kC));
    c.omega = cfg->lambda > 0 ? 2.0 * kPi * kC / cfg->lambda : 0.0;
    const double Lant = (double)(c.k_ant - cfg->slab_k) * cfg->dx;
    c.t_ant = cfg->t_peak - Lant / kC;
    // workspace
    Carver cv{(char*)workspace, (char*)workspace + workspace_bytes};
    for (int s = 0; s < 2; s++) {
        Species& S = c.sp[s];
        memset(&S, 0, sizeof(S));
        SpeciesBuf* bufs[2] = {&S.a, &S.b};
        for (int b = 0; b < 2; b++) {
            bufs[b]->cell = cv.take<int32_t>(L.cap[s]);
            bufs[b]->fx = cv.take<float>(L.cap[s]);
            bufs[b]->fy = d3 ? cv.take<float>(L.cap[s]) : nullptr;
            bufs[b]->fz = cv.take<float>(L.cap[s]);
            bufs[b]->ux = cv.take<float>(L.cap[s]);
            bufs[b]->uy = cv.take<float>(L.cap[s]);
            bufs[b]->uz = cv.take<float>(L.cap[s]);
        }
        S.tile_start = cv.take<int32_t>(L.ntiles + 1);
        S.n = L.n0[s];
        S.cap = L.cap[s];
    }
    for (int q = 0; q < 6; q++) c.F[q] = cv.take<float>(L.nn);
    for (int q = 0; q < 3; q++) c.J[q] = cv.take<u64>(L.nn);
    for (int q = 0; q < 2; q++) c.rho[q] = cv.take<u64>(L.nn);
    const size_t plane = (size_t)L.nx * L.ny;
    c.mur_save = cv.take<float>(8 * plane);
    c.ant_c = cv.take<float>(plane);
    c.ant_s = cv.take<float>(plane);
    c.ant = cv.take<float>(2);
    c.keys_count = cv.take<int32_t>((size_t)L.nkeys + 1);
    c.keys_off = cv.take<int32_t>((size_t)L.nkeys + 1);
    c.scan_tmp = cv.take<int32_t>(((size_t)L.nkeys + 2047) / 2048 + 1);
    c.partials = cv.take<double>(5 * (size_t)kMaxEnergyBlocks);
    c.red_out = cv.take<double>(8);
    c.status = cv.take<unsigned>(8);
    if (cv.p > cv.end) {
        delete h;
        return PIC_ENOMEM;
    }
    if (energy_blocks(c) > kMaxEnergyBlocks) {
        delete h;
        return PIC_EINVAL;
    }
    // species constants
    const double mi = cfg->ion_mass_amu * kAmu;
    const double qi = cfg->ion_charge * kQe;
    const double uth_i = sqrt(kKb * cfg->T_ion_K / (mi * kC * kC));
    const double uth_e = sqrt(cfg->T_electron_eV * kQe / (kMe * kC * kC));
    const double qs[2] = {qi, -kQe}, ms[2] = {mi, kMe}, uths[2] = {uth_i, uth_e};
    for (int s = 0; s < 2; s++) {
        Species& S = c.sp[s];
        S.ppc = s == 0 ? cfg->ppc_ion : cfg->ppc_electron;
        S.mass = ms[s];
        S.uth = uths[s];
        S.e_kick = (float)(qs[s] * c.dt / (2.0 * ms[s] * kC));
        S.b_rot = (float)(qs[s] * c.dt / (2.0 * ms[s]));
        S.pair = s == 0;
        S.p_kick = S.pair ? (float)(c.dt * (c.D / c.r0) / (2.0 * ms[s] * kC)) : 0.0f;
        S.jsign = (cfg->mode == PIC_MODE_FULL) ? (s == 0 ? 1 : -1) : 0;
    }
    // antenna table (x = i + 1/2, FP64 -> FP32)
    {
        // paraxial Gaussian beam converging on the slab surface, evaluated at the antenna: width w_a,
        // curvature R_a, Gouy phase (half of it for a 2D line focus), amplitude (w0/w_a)^(1/2) in 2D,
        // w0/w_a in 3D; E_x sits at (i + 1/2, j)
        std::vector<float> ac(plane, 0.f), as(plane, 0.f);
        if (cfg->laser_profile == PIC_LASER_PLANE) {
            for (size_t q = 0; q < plane; q++) ac[q] = 1.0f;
        } else if (cfg->laser_profile == PIC_LASER_GAUSSIAN) {
            const double zR = kPi * cfg->w0 * cfg->w0 / cfg->lambda, sa = -Lant;
            const double wa = cfg->w0 * sqrt(1.0 + (sa / zR) * (sa / zR));
            const double Ra = sa + zR * zR / sa;
            const double gouy = (d3 ? 1.0 : 0.5) * atan(sa / zR);
            const double amp0 = d3 ? cfg->w0 / wa : sqrt(cfg->w0 / wa);
            const double kw = c.omega / kC;
            for (int j = 0; j < L.ny; j++)
                for (int i = 0; i < L.nx; i++) {
                    const double xr = ((double)i + 0.5 - 0.5 * L.nx) * cfg->dx;
                    const double yr = d3 ? ((double)j - 0.5 * L.ny) * cfg->dx : 0.0;
                    const double r2 = xr * xr + yr * yr;
                    const double amp = amp0 * exp(-r2 / (wa * wa));
                    const double ph = -kw * r2 / (2.0 * Ra) + gouy;
                    ac[(size_t)j * L.nx + i] = (float)(amp * cos(ph));
                    as[(size_t)j * L.nx + i] = (float)(amp * sin(ph));
                }
        }
        if (cudaMemcpyAsync(c.ant_c, ac.data(), 4 * plane, cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
            cudaMemcpyAsync(c.ant_s, as.data(), 4 * plane, cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
            cudaStreamSynchronize(c.stream) != cudaSuccess) {
            delete h;
            return PIC_ECUDA;
        }
    }
    bool ok = true;
    for (int q = 0; q < 6; q++) ok &= cudaMemsetAsync(c.F[q], 0, 4 * L.nn, c.stream) == cudaSuccess;
    for (int q = 0; q < 3; q++) ok &= cudaMemsetAsync(c.J[q], 0, 8 * L.nn, c.stream) == cudaSuccess;
    for (int q = 0; q < 2; q++) ok &= cudaMemsetAsync(c.rho[q], 0, 8 * L.nn, c.stream) == cudaSuccess;
    ok &= cudaMemsetAsync(c.mur_save, 0, 4 * 8 * plane, c.stream) == cudaSuccess;
    ok &= cudaMemsetAsync(c.red_out, 0, 8 * sizeof(double), c.stream) == cudaSuccess;   // incl. the injected-energy sum
    ok &= cudaMemsetAsync(c.status, 0, 32, c.stream) == cudaSuccess;
    if (!ok) {
        delete h;
        return PIC_ECUDA;
    }
    c.cur = 0;
    // initial particles into the second buffers, then sort into tiles
    for (int s = 0; s < c.nsp; s++) {
        if (d3) launch_init_particles3(c, s, c.stream);
        else launch_init_particles(c, s, c.stream);
        sort_species_impl(c, s, c.stream, 1, nullptr);
    }
    r = redeposit(c);
    if (r == PIC_OK && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c.stream) != cudaSuccess))
        r = PIC_ECUDA;
    if (r) {
        delete h;
        return r;
    }
    *out = h;
    return PIC_OK;
}

void pic_free(pic_ctx* h)
{
    if (!h) return;
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    delete h;
}

int pic_step(pic_ctx* h, int32_t nsteps)
{
    if (!h || nsteps < 0) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.in_batch) return PIC_ESTATE;
    if (c.sticky) return c.sticky;
    for (int it = 0; it < nsteps; it++) {
        if (c.cfg.sort_every > 0 && c.steps_since_sort >= c.cfg.sort_every) {
            int r = sort_all(h);
            if (r) return r;
        }
        {
            // clear the currents; the next node density starts from the current one (the particle
            // kernel adds the changes)
            const CopySeg prep[4] = {{nullptr, c.J[0], 8 * c.nn}, {nullptr, c.J[1], 8 * c.nn},
                                     {nullptr, c.J[2], 8 * c.nn}, {c.rho[c.cur], c.rho[1 - c.cur], 8 * c.nn}};
            c.nlaunch[3] += launch_copy_segments(c, prep, 4, c.stream);
            CK(cudaGetLastError());
        }
        int r = ev_begin(h, 0);
        if (r) return r;
        if (c.dims == 3) launch_particle_step3(c, c.stream);
        else launch_particle_step(c, make_step_args(c), c.stream);
        r = ev_end(h);
        if (r) return r;
        c.nlaunch[0]++;
        c.nlaunch[3]++;
        if (c.cfg.mode == PIC_MODE_FULL) {
            r = ev_begin(h, 1);
            if (r) return r;
            const int64_t before = c.nlaunch[1];
            if (c.dims == 3) launch_fields3(c, c.stream, c.step, &c.nlaunch[1]);
            else launch_fields(c, c.stream, c.step, &c.nlaunch[1]);
            r = ev_end(h);
            if (r) return r;
            c.nlaunch[3] += c.nlaunch[1] - before;
        }
        CK(cudaGetLastError());
        c.cur = 1 - c.cur;
        c.step++;
        c.steps_since_sort++;
    }
    return finish_status(h);
}

int pic_deposit_density(pic_ctx* h, int64_t* dev_out, double* scale_out)
{
    if (!h || !dev_out) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.sticky) return c.sticky;
    if (c.dims == 3) launch_deposit_density3(c, (u64*)dev_out, c.stream);
    else launch_deposit_density(c, (u64*)dev_out, c.stream);
    CK(cudaGetLastError());
    if (scale_out)
        *scale_out = c.dims == 3 ? c.w / (4398046511104.0 * c.cfg.dx * c.cfg.dx * c.cfg.dx)
                                 : c.w / (4294967296.0 * c.cfg.dx * c.cfg.dx);
    return PIC_OK;
}

int pic_pair_force_at(pic_ctx* h, int64_t n, const int32_t* dev_cell, const float* dev_fx, const float* dev_fz,
                      int32_t pot_mode, double c_att, double s_rep, float* dev_out)
{
    if (!h || n < 0 || (n > 0 && (!dev_cell || !dev_fx || !dev_fz || !dev_out))) return PIC_EINVAL;
    if (pot_mode < 0 || pot_mode > 2) return PIC_EINVAL;
    Ctx& c = h->c;
    if (pot_mode == 2 && !(c.cfg.morse_a > 0 && c.cfg.morse_a < 1e3)) return PIC_EINVAL;
    if (pot_mode == 2) c_att = c.cfg.morse_a;
    if (c.dims == 3) return PIC_ESTATE;
    if (c.sticky) return c.sticky;
    launch_pair_force_probe(c, n, dev_cell, dev_fx, dev_fz, pot_mode | (pot_code(c.cfg) & 4), c_att, s_rep, dev_out,
                            c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

int pic_cell_temperature(pic_ctx* h, int32_t species, double* dev_work, double* dev_T)
{
    if (!h || !dev_work || !dev_T) return PIC_EINVAL;
    Ctx& c = h->c;
    if (species < 0 || species >= c.nsp) return PIC_EINVAL;
    if (c.sticky) return c.sticky;
    launch_cell_temperature(c, species, dev_work, dev_T, c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

int pic_set_temperature(pic_ctx* h, int32_t species, const double* dev_T, double T_from)
{
    if (!h || !dev_T || !(T_from > 0)) return PIC_EINVAL;
    Ctx& c = h->c;
    if (species < 0 || species >= c.nsp) return PIC_EINVAL;
    if (c.sticky) return c.sticky;
    launch_set_temperature(c, species, dev_T, T_from, c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

int pic_crater_profile(pic_ctx* h, const int64_t* dev_rho0, double* dev_out)
{
    if (!h || !dev_rho0 || !dev_out) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.sticky) return c.sticky;
    const double scale = c.dims == 3 ? c.w / (4398046511104.0 * c.cfg.dx * c.cfg.dx * c.cfg.dx)
                                     : c.w / (4294967296.0 * c.cfg.dx * c.cfg.dx);
    launch_crater_profile(c, (const u64*)dev_rho0, c.cfg.dx * scale / c.cfg.n_atoms, dev_out, c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

int pic_pair_force(pic_ctx* h, float* dev_out)
{
    if (!h || !dev_out) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.sticky) return c.sticky;
    if (c.dims == 3) launch_pair_force3(c, dev_out, c.stream);
    else launch_pair_force(c, dev_out, c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

int pic_energy(pic_ctx* h, pic_energy_t* out)
{
    if (!h || !out) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.sticky) return c.sticky;
    double e[5];
    if (c.dims == 3) launch_energy3(c, c.stream, e);
    else launch_energy(c, c.stream, e);
    CK(cudaGetLastError());
    out->kinetic_ion = e[0];
    out->kinetic_electron = e[1];
    out->field_E = e[2];
    out->field_B = e[3];
    out->pair = e[4];
    out->step = c.step;
    // injected energy: -sum (Ex By - Ey Bx) / mu0 * (cell edge, or area in 3D) * dt
    double flux = 0.0;
    CK(cudaMemcpyAsync(&flux, c.red_out + 5, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    const double mu0 = 1.0 / (kEps0 * kC * kC);
    out->injected = -flux / mu0 * c.cfg.dx * (c.dims == 3 ? c.cfg.dx : 1.0) * c.dt;
    return PIC_OK;
}

int pic_get_info(pic_ctx* h, pic_info* out)
{
    if (!h || !out) return PIC_EINVAL;
    const Ctx& c = h->c;
    out->dt = c.dt;
    out->weight = c.w;
    out->rho_scale = c.rho_scale;
    out->r0 = c.r0;
    out->time = (double)c.step * c.dt;
    out->step = c.step;
    out->num_particles[0] = c.sp[0].n;
    out->num_particles[1] = c.nsp > 1 ? c.sp[1].n : 0;
    out->nspecies = c.nsp;
    out->ntiles = c.ntiles;
    return PIC_OK;
}

static cudaMemcpyKind kind_out(int32_t on_host) { return on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }
static cudaMemcpyKind kind_in(int32_t on_host) { return on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }

int pic_get_particles(pic_ctx* h, int32_t s, int32_t* cell, float* fx, float* fy, float* fz, float* ux, float* uy,
                      float* uz, int32_t on_host)
{
    if (!h || s < 0 || s >= h->c.nsp) return PIC_EINVAL;
    Ctx& c = h->c;
    const Species& S = c.sp[s];
    const size_t n = (size_t)S.n;
    if (n == 0) return PIC_OK;
    if (!cell || !fx || !fz || !ux || !uy || !uz || (c.dims == 3 && !fy)) return PIC_EINVAL;
    CK(cudaMemcpyAsync(cell, S.a.cell, 4 * n, kind_out(on_host), c.stream));
    CK(cudaMemcpyAsync(fx, S.a.fx, 4 * n, kind_out(on_host), c.stream));
    if (c.dims == 3) CK(cudaMemcpyAsync(fy, S.a.fy, 4 * n, kind_out(on_host), c.stream));
    CK(cudaMemcpyAsync(fz, S.a.fz, 4 * n, kind_out(on_host), c.stream));
    CK(cudaMemcpyAsync(ux, S.a.ux, 4 * n, kind_out(on_host), c.stream));
    CK(cudaMemcpyAsync(uy, S.a.uy, 4 * n, kind_out(on_host), c.stream));
    CK(cudaMemcpyAsync(uz, S.a.uz, 4 * n, kind_out(on_host), c.stream));
    if (on_host) CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_set_particles(pic_ctx* h, int32_t s, int64_t n, const int32_t* cell, const float* fx, const float* fy,
                      const float* fz, const float* ux, const float* uy, const float* uz, int32_t on_host)
{
    if (!h || s < 0 || s >= h->c.nsp || n < 0) return PIC_EINVAL;
    Ctx& c = h->c;
    Species& S = c.sp[s];
    if (n > S.cap) return PIC_ENOMEM;
    if (n > 0 && (!cell || !fx || !fz || !ux || !uy || !uz || (c.dims == 3 && !fy))) return PIC_EINVAL;
    const size_t b = 4 * (size_t)n;
    if (n > 0) {
        CK(cudaMemcpyAsync(S.b.cell, cell, b, kind_in(on_host), c.stream));
        CK(cudaMemcpyAsync(S.b.fx, fx, b, kind_in(on_host), c.stream));
        if (c.dims == 3) CK(cudaMemcpyAsync(S.b.fy, fy, b, kind_in(on_host), c.stream));
        CK(cudaMemcpyAsync(S.b.fz, fz, b, kind_in(on_host), c.stream));
        CK(cudaMemcpyAsync(S.b.ux, ux, b, kind_in(on_host), c.stream));
        CK(cudaMemcpyAsync(S.b.uy, uy, b, kind_in(on_host), c.stream));
        CK(cudaMemcpyAsync(S.b.uz, uz, b, kind_in(on_host), c.stream));
        // reject cells outside the grid and offsets outside the cell before any kernel uses them
        unsigned* bad = c.status + 1;
        CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), c.stream));
        launch_validate(c, S.b, n, bad, c.stream);
        CK(cudaGetLastError());
        unsigned hbad = 0;
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
        if (hbad) return PIC_EINVAL;
    }
    S.n = n;
    sort_species_impl(c, s, c.stream, 1, nullptr);
    CK(cudaGetLastError());
    if (s == 0) {
        int r = redeposit(c);
        if (r) return r;
    }
    CK(cudaStreamSynchronize(c.stream));
    c.steps_since_sort = 0;
    return PIC_OK;
}

int pic_get_field(pic_ctx* h, int32_t which, float* out, int32_t on_host)
{
    if (!h || which < 0 || which > 5 || !out) return PIC_EINVAL;
    Ctx& c = h->c;
    CK(cudaMemcpyAsync(out, c.F[which], 4 * c.nn, kind_out(on_host), c.stream));
    if (on_host) CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_set_field(pic_ctx* h, int32_t which, const float* in, int32_t on_host)
{
    if (!h || which < 0 || which > 5 || !in) return PIC_EINVAL;
    Ctx& c = h->c;
    CK(cudaMemcpyAsync(c.F[which], in, 4 * c.nn, kind_in(on_host), c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_get_current(pic_ctx* h, int64_t* out3, int32_t on_host)
{
    if (!h || !out3) return PIC_EINVAL;
    Ctx& c = h->c;
    for (int q = 0; q < 3; q++)
        CK(cudaMemcpyAsync(out3 + q * c.nn, c.J[q], 8 * c.nn, kind_out(on_host), c.stream));
    if (on_host) CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_get_density(pic_ctx* h, int64_t* out, int32_t on_host)
{
    if (!h || !out) return PIC_EINVAL;
    Ctx& c = h->c;
    CK(cudaMemcpyAsync(out, c.rho[c.cur], 8 * c.nn, kind_out(on_host), c.stream));
    if (on_host) CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_sort(pic_ctx* h)
{
    if (!h) return PIC_EINVAL;
    int r = sort_all(h);
    if (r) return r;
    CK(cudaStreamSynchronize(h->c.stream));
    return PIC_OK;
}

int pic_set_timing(pic_ctx* h, int32_t enable)
{
    if (!h) return PIC_EINVAL;
    Ctx& c = h->c;
    c.timing = enable != 0;
    for (int q = 0; q < 3; q++) c.ms[q] = 0.0;
    for (int q = 0; q < 4; q++) c.nlaunch[q] = 0;
    h->evkind.clear();
    return PIC_OK;
}

int pic_get_timing(pic_ctx* h, double ms[3], int64_t n[4])
{
    if (!h || !ms || !n) return PIC_EINVAL;
    for (int q = 0; q < 3; q++) ms[q] = h->c.ms[q];
    for (int q = 0; q < 4; q++) n[q] = h->c.nlaunch[q];
    return PIC_OK;
}

// ---- checkpoint / resume ---------------------------------------------------------------------

namespace {

struct CkptHeader {
    int64_t magic, step, n[2];
    int32_t steps_since_sort, nsp;
};
constexpr int64_t kCkptMagic = 0x504943434b505431LL;

size_t ckpt_layout(const Ctx& c, size_t* off_sp, size_t* off_tiles, size_t* off_f, size_t* off_rho, size_t* off_j)
{
    size_t t = align256(sizeof(CkptHeader));
    const int arrays = c.dims == 3 ? 7 : 6;
    for (int s = 0; s < 2; s++) {
        off_sp[s] = t;
        t += arrays * align256(4 * (size_t)(c.sp[s].cap > 0 ? c.sp[s].cap : 1));
        off_tiles[s] = t;
        t += align256(4 * (size_t)(c.ntiles + 1));
    }
    *off_f = t;
    t += 6 * align256(4 * c.nn);
    *off_rho = t;
    t += align256(8 * c.nn);
    *off_j = t;
    t += 3 * align256(8 * c.nn);
    t += align256(sizeof(double));      // the injected-energy sum
    return t;
}

int ckpt_copy(pic_ctx* h, char* buf, bool save, bool on_host)
{
    Ctx& c = h->c;
    size_t osp[2], otl[2], of, orho, oj;
    ckpt_layout(c, osp, otl, &of, &orho, &oj);
    const cudaMemcpyKind k = save ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
    // device buffers: all segments in one vectorised copy kernel; host buffers: one copy each
    std::vector<CopySeg> segs;
    auto cp = [&](void* dev, size_t off, size_t bytes) -> cudaError_t {
        if (!on_host) {
            segs.push_back(save ? CopySeg{dev, buf + off, bytes} : CopySeg{buf + off, dev, bytes});
            return cudaSuccess;
        }
        return save ? cudaMemcpyAsync(buf + off, dev, bytes, k, c.stream) : cudaMemcpyAsync(dev, buf + off, bytes, k, c.stream);
    };
    for (int s = 0; s < c.nsp; s++) {
        Species& S = c.sp[s];
        const size_t b = 4 * (size_t)S.n, slot = align256(4 * (size_t)S.cap);
        void* arr[7] = {S.a.cell, S.a.fx, S.a.fz, S.a.ux, S.a.uy, S.a.uz, S.a.fy};
        const int arrays = c.dims == 3 ? 7 : 6;
        for (int q = 0; q < arrays; q++)
            if (b) CK(cp(arr[q], osp[s] + q * slot, b));
        CK(cp(S.tile_start, otl[s], 4 * (size_t)(c.ntiles + 1)));
    }
    for (int q = 0; q < 6; q++) CK(cp(c.F[q], of + q * align256(4 * c.nn), 4 * c.nn));
    CK(cp(c.rho[c.cur], orho, 8 * c.nn));
    for (int q = 0; q < 3; q++) CK(cp(c.J[q], oj + q * align256(8 * c.nn), 8 * c.nn));
    CK(cp(c.red_out + 5, oj + 3 * align256(8 * c.nn), sizeof(double)));
    if (!on_host) {
        launch_copy_segments(c, segs.data(), (int)segs.size(), c.stream);
        CK(cudaGetLastError());
    }
    return PIC_OK;
}

}  // namespace

int pic_checkpoint_size(pic_ctx* h, size_t* bytes)
{
    if (!h || !bytes) return PIC_EINVAL;
    size_t osp[2], otl[2], of, orho, oj;
    *bytes = ckpt_layout(h->c, osp, otl, &of, &orho, &oj);
    return PIC_OK;
}

int pic_checkpoint_save(pic_ctx* h, void* buf, int32_t on_host)
{
    if (!h || !buf || (!on_host && ((uintptr_t)buf & 255))) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.sticky) return c.sticky;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = kCkptMagic;
    hd.step = c.step;
    hd.n[0] = c.sp[0].n;
    hd.n[1] = c.nsp > 1 ? c.sp[1].n : 0;
    hd.steps_since_sort = c.steps_since_sort;
    hd.nsp = c.nsp;
    if (on_host) {
        memcpy(buf, &hd, sizeof(hd));
        int r = ckpt_copy(h, (char*)buf, true, true);
        if (r) return r;
        CK(cudaStreamSynchronize(c.stream));             // the host copy is complete on return
        return PIC_OK;
    }
    // a pageable source: the call returns once the header has been staged, so hd may go out of scope
    CK(cudaMemcpyAsync(buf, &hd, sizeof(hd), cudaMemcpyHostToDevice, c.stream));
    return ckpt_copy(h, (char*)buf, true, false);
}

int pic_checkpoint_restore(pic_ctx* h, const void* buf, int32_t on_host)
{
    if (!h || !buf || (!on_host && ((uintptr_t)buf & 255))) return PIC_EINVAL;
    Ctx& c = h->c;
    CkptHeader hd;
    if (on_host) {
        memcpy(&hd, buf, sizeof(hd));
    } else {
        CK(cudaMemcpyAsync(&hd, buf, sizeof(hd), cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    if (hd.magic != kCkptMagic || hd.nsp != c.nsp) return PIC_EINVAL;
    for (int s = 0; s < c.nsp; s++)
        if (hd.n[s] < 0 || hd.n[s] > c.sp[s].cap) return PIC_EINVAL;
    for (int s = 0; s < c.nsp; s++) c.sp[s].n = hd.n[s];
    int r = ckpt_copy(h, (char*)const_cast<void*>(buf), false, on_host != 0);
    if (r) return r;
    c.step = hd.step;
    c.steps_since_sort = hd.steps_since_sort;
    CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

// ---- differentiable transport stage -------------------------------------------------------

static int adjoint_ok(const Ctx& c, const pic_adjoint_buffers* b)
{
    if (c.sticky) return c.sticky;
    if (c.dims != 2 || c.cfg.sort_every != 0 || c.cfg.pot_mode != 0 || c.cfg.lattice != 0) return PIC_ESTATE;
    for (int s = 0; s < c.nsp; s++)
        if (!b->lam_pos[s] || !b->lam_u[s]) return PIC_EINVAL;
    if (!b->lam_nodes || !b->grads) return PIC_EINVAL;
    if (c.cfg.mode == PIC_MODE_FULL && (!b->lam_F || !b->lam_j)) return PIC_EINVAL;
    return PIC_OK;
}

int pic_node_functional(pic_ctx* h, const double* dev_weights, double* host_out)
{
    if (!h || !dev_weights || !host_out) return PIC_EINVAL;
    Ctx& c = h->c;
    if (c.dims != 2) return PIC_ESTATE;
    double* tmp = c.red_out + 7;
    launch_node_functional(c, dev_weights, tmp, c.stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_out, tmp, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_adjoint_seed(pic_ctx* h, double kin, const double* dev_weights, const pic_adjoint_buffers* b,
                     double* host_dLdr0)
{
    if (!h || !dev_weights || !b || !host_dLdr0) return PIC_EINVAL;
    Ctx& c = h->c;
    int r = adjoint_ok(c, b);
    if (r) return r;
    double* tmp = c.red_out + 6;
    CK(cudaMemsetAsync(tmp, 0, sizeof(double), c.stream));
    if (c.cfg.mode == PIC_MODE_FULL)
        launch_adjoint_seed_full(c, kin, dev_weights, b->lam_pos, b->lam_u, b->lam_nodes, b->lam_F, b->lam_j, tmp,
                                 c.stream);
    else
        launch_adjoint_seed(c, kin, dev_weights, b->lam_pos[0], b->lam_u[0], b->lam_nodes, tmp, c.stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_dLdr0, tmp, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return PIC_OK;
}

int pic_adjoint_step(pic_ctx* h, const pic_adjoint_buffers* b)
{
    if (!h || !b) return PIC_EINVAL;
    Ctx& c = h->c;
    int r = adjoint_ok(c, b);
    if (r) return r;
    if (c.cfg.mode == PIC_MODE_FULL)
        launch_adjoint_step_full(c, b->lam_pos, b->lam_u, b->lam_nodes, b->lam_F, b->lam_j, b->grads, c.stream);
    else
        launch_adjoint_step(c, b->lam_pos[0], b->lam_u[0], b->lam_nodes, b->grads, c.stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

const char* pic_strerror(int code)
{
    switch (code) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "workspace too small or particle count above capacity";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_ENAN: return "non-finite particle momentum";
    case PIC_EMOVE: return "a particle moved one cell or more in one step";
    case PIC_ESTATE: return "operation not valid in this mode";
    case PIC_EOVERFLOW: return "a fixed-point node sum could overflow int64 for this configuration";

    default: return "unknown error";
    }
}

}  // extern "C"
