// Reverse-mode (adjoint) kernels of the 2D cycle, for gradients of a loss of the final state with
// respect to the pair-potential parameters D and r0 (r0 sets Eq. (3)'s equilibrium distance, the
// r0/dx of Eq. (1), and the density unit n0 = r0^-3) and, with fields, the laser peak intensity.
//
// Part 1: the atomic-transport stage (neutral atoms, pair force only; paper: the transport
// simulation evolves the target with the pair potential).
//
// Forward step (per atom): node density n(x) -> gather (n, dn/dxi, dn/dzeta) -> force F(n, q) of
// Eqs. (1)-(3) -> u += F dt / (m c) -> x += c dt u / (gamma dx) -> wall mirror.
// The adjoint treats the fixed-point deposition as the continuous linear shape (straight-through)
// and runs in FP64. One reverse step (adjoint kernels A and B) maps the adjoints of
// (x^(t+1), u^(t+1)) to those of (x^t, u^t) and accumulates the parameter gradients:
//   A: per atom -- transpose of the position update and of the kick, force derivatives, the
//      gather's position derivatives, and the gather's transpose onto the nodes (FP64 atomics);
//   B: per atom -- transpose of the deposition: the node adjoints' interpolated gradient.
#include "pic_device.cuh"

namespace gbpic {

struct AdjArgs {
    int nx, nz;
    unsigned nx_magic;
    int64_t n;
    const int32_t* cell;
    const float *fx, *fz, *ux, *uy, *uz;
    const u64* rho;        // fixed-point node sums at the current positions
    double rho_s;          // node sum -> n / n0
    double unit;           // one atom's full weight on a node, in units of n0 (rho_s * 2^32)
    double D, r0, dx, kick, cs0;   // kick = dt / (m c); cs0 = c dt / dx
    double* lam_pos;       // 2 n: (x, z) adjoints, per cell
    double* lam_u;         // 3 n
    double* lam_nodes;     // (nz + 1) nx node adjoints (units 1 / n0)
    double* grads;         // 2: dL/dD, dL/dr0
};

__device__ __forceinline__ double node_n(const AdjArgs& a, int i, int k)
{
    const long long v = (long long)a.rho[(size_t)k * a.nx + i];
    return a.rho_s * (double)((k == 0 || k == a.nz) ? 2 * v : v);
}

// F (N) and partial derivatives along one axis from (n, q), Eqs. (1)-(3)
__device__ __forceinline__ double axis_force_d(double n, double q, double D, double r0, double dx, double& dFdn,
                                               double& dFdq, double& dFdr0)
{
    dFdn = dFdq = dFdr0 = 0.0;
    if (!(n > 0.0)) return 0.0;
    const double c = cbrt(n);                     // n^(1/3)
    const double rbar = 1.0 / c;
    const double n43 = 1.0 / (n * c);             // n^(-4/3)
    const double h = -(1.0 / 6.0) * (r0 / dx) * n43 * q;
    const double drbar_dn = -(1.0 / 3.0) * n43;
    const double dh_dn = (2.0 / 9.0) * (r0 / dx) * n43 / n * q;
    const double dh_dq = -(1.0 / 6.0) * (r0 / dx) * n43;
    const double fu = D / r0;
    double F = 0.0, dF_drbar = 0.0, dF_dh = 0.0;
    if (1.0 - h > 0.0) {
        const double ia = c * (1.0 - h), i2 = ia * ia, i6 = i2 * i2 * i2, i7 = i6 * ia, i8 = i6 * i2;
        const double up = 12.0 * i7 * (1.0 - i6), upp = i8 * (156.0 * i6 - 84.0);
        F += fu * up;
        dF_drbar += fu * upp / (1.0 - h);
        dF_dh += fu * upp * rbar / ((1.0 - h) * (1.0 - h));
    }
    if (1.0 + h > 0.0) {
        const double ib = c * (1.0 + h), i2 = ib * ib, i6 = i2 * i2 * i2, i7 = i6 * ib, i8 = i6 * i2;
        const double up = 12.0 * i7 * (1.0 - i6), upp = i8 * (156.0 * i6 - 84.0);
        F -= fu * up;
        dF_drbar -= fu * upp / (1.0 + h);
        dF_dh += fu * upp * rbar / ((1.0 + h) * (1.0 + h));
    }
    dFdn = dF_drbar * drbar_dn + dF_dh * dh_dn;
    dFdq = dF_dh * dh_dq;
    dFdr0 = -F / r0 + dF_dh * h / r0;
    return F;
}

__device__ __forceinline__ void split2(int cell, int nx, unsigned magic, int& i, int& k)
{
    unsigned q = __umulhi((unsigned)cell, magic);
    int r = cell - (int)q * nx;
    if (r >= nx) { q++; r -= nx; }
    k = (int)q;
    i = r;
}

__device__ __forceinline__ double block_sum_d(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_adjoint_a(const AdjArgs a)
{
    __shared__ double sh[256];
    double gD = 0.0, gR = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        int i, k;
        split2(a.cell[p], a.nx, a.nx_magic, i, k);
        double fx = a.fx[p], fz = a.fz[p];
        if (k >= a.nz) { k = a.nz - 1; fz = 1.0; }
        const int i1 = i + 1 == a.nx ? 0 : i + 1;
        const double n00 = node_n(a, i, k), n10 = node_n(a, i1, k), n01 = node_n(a, i, k + 1), n11 = node_n(a, i1, k + 1);
        const double n = (1 - fx) * (1 - fz) * n00 + fx * (1 - fz) * n10 + (1 - fx) * fz * n01 + fx * fz * n11;
        const double qx = (1 - fz) * (n10 - n00) + fz * (n11 - n01);
        const double qz = (1 - fx) * (n01 - n00) + fx * (n11 - n10);
        const double gxz = n11 - n01 - n10 + n00;
        double dxn, dxq, dxr, dzn, dzq, dzr;
        const double Fx = axis_force_d(n, qx, a.D, a.r0, a.dx, dxn, dxq, dxr);
        const double Fz = axis_force_d(n, qz, a.D, a.r0, a.dx, dzn, dzq, dzr);
        // forward quantities of this step: kicked momentum (before the wall mirror), move
        const double ux = (double)a.ux[p] + a.kick * Fx, uy = (double)a.uy[p], uz = (double)a.uz[p] + a.kick * Fz;
        const double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz), cs = a.cs0 / g;
        const double zn = (double)k + fz + uz * cs;
        const bool refl = zn < 0.0 || zn >= (double)a.nz;
        double lpx = a.lam_pos[2 * p], lpz = a.lam_pos[2 * p + 1];
        double lux = a.lam_u[3 * p], luy = a.lam_u[3 * p + 1], luz = a.lam_u[3 * p + 2];
        if (refl) { lpz = -lpz; luz = -luz; }
        // position update x' = x + cs u: dx'/du = cs (I - u u^T / gamma^2)
        const double udl = (ux * lpx + uz * lpz) / (g * g);
        lux += cs * (lpx - ux * udl);
        luy += cs * (0.0 - uy * udl);
        luz += cs * (lpz - uz * udl);
        // kick u' = u + kick F
        const double lFx = a.kick * lux, lFz = a.kick * luz;
        gD += (lFx * Fx + lFz * Fz) / a.D;
        gR += lFx * (dxr + dxn * 3.0 * n / a.r0 + dxq * 3.0 * qx / a.r0) +
              lFz * (dzr + dzn * 3.0 * n / a.r0 + dzq * 3.0 * qz / a.r0);
        const double ln = lFx * dxn + lFz * dzn, lqx = lFx * dxq, lqz = lFz * dzq;
        a.lam_pos[2 * p] = lpx + ln * qx + lqz * gxz;
        a.lam_pos[2 * p + 1] = lpz + ln * qz + lqx * gxz;
        a.lam_u[3 * p] = lux;
        a.lam_u[3 * p + 1] = luy;
        a.lam_u[3 * p + 2] = luz;
        // transpose of the gather onto the four corners
        double* L0 = a.lam_nodes + (size_t)k * a.nx;
        double* L1 = L0 + a.nx;
        atomicAdd(L0 + i, ln * (1 - fx) * (1 - fz) - lqx * (1 - fz) - lqz * (1 - fx));
        atomicAdd(L0 + i1, ln * fx * (1 - fz) + lqx * (1 - fz) - lqz * fx);
        atomicAdd(L1 + i, ln * (1 - fx) * fz - lqx * fz + lqz * (1 - fx));
        atomicAdd(L1 + i1, ln * fx * fz + lqx * fz + lqz * fx);
    }
    const double sD = block_sum_d(gD, sh), sR = block_sum_d(gR, sh);
    if (threadIdx.x == 0) {
        atomicAdd(a.grads, sD);
        atomicAdd(a.grads + 1, sR);
    }
}

// lam_pos += d/dx of sum_nodes lam_nodes * n^(nodes) (transpose of the deposition)
__global__ void k_adjoint_b(const AdjArgs a)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        int i, k;
        split2(a.cell[p], a.nx, a.nx_magic, i, k);
        double fx = a.fx[p], fz = a.fz[p];
        if (k >= a.nz) { k = a.nz - 1; fz = 1.0; }
        const int i1 = i + 1 == a.nx ? 0 : i + 1;
        const double m0 = k == 0 ? 2.0 : 1.0, m1 = k + 1 == a.nz ? 2.0 : 1.0;
        const double* L0 = a.lam_nodes + (size_t)k * a.nx;
        const double* L1 = L0 + a.nx;
        const double l00 = m0 * L0[i], l10 = m0 * L0[i1], l01 = m1 * L1[i], l11 = m1 * L1[i1];
        a.lam_pos[2 * p] += a.unit * ((1 - fz) * (l10 - l00) + fz * (l11 - l01));
        a.lam_pos[2 * p + 1] += a.unit * ((1 - fx) * (l01 - l00) + fx * (l11 - l10));
    }
}

// seed: lam_u = kin * w m c^2 u / gamma; sum of lam_nodes * 3 n / r0 (the density unit's r0 dependence)
__global__ void __launch_bounds__(256) k_adjoint_seed(const AdjArgs a, double kin_mc2w, const double* w_nodes,
                                                      int64_t nn, double* r0_out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        const double ux = a.ux[p], uy = a.uy[p], uz = a.uz[p];
        const double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        a.lam_u[3 * p] = kin_mc2w * ux / g;
        a.lam_u[3 * p + 1] = kin_mc2w * uy / g;
        a.lam_u[3 * p + 2] = kin_mc2w * uz / g;
        a.lam_pos[2 * p] = 0.0;
        a.lam_pos[2 * p + 1] = 0.0;
    }
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nn; c += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / a.nx), i = (int)(c - (int64_t)k * a.nx);
        acc += w_nodes[c] * 3.0 * node_n(a, i, k) / a.r0;
    }
    const double s = block_sum_d(acc, sh);
    if (threadIdx.x == 0) atomicAdd(r0_out, s);
}

// value of sum_nodes w * n^
__global__ void __launch_bounds__(256) k_node_functional(const u64* rho, int nx, int nz, double rho_s, const double* w,
                                                         int64_t nn, double* out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nn; c += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / nx);
        const long long v = (long long)rho[c];
        acc += w[c] * rho_s * (double)((k == 0 || k == nz) ? 2 * v : v);
    }
    const double s = block_sum_d(acc, sh);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

static AdjArgs make_adj(Ctx& c, double* lam_pos, double* lam_u, double* lam_nodes, double* grads)
{
    AdjArgs a;
    a.nx = c.nx;
    a.nz = c.nz;
    a.nx_magic = (unsigned)(4294967296ULL / (unsigned long long)c.nx);
    const Species& S = c.sp[0];
    a.n = S.n;
    a.cell = S.a.cell;
    a.fx = S.a.fx;
    a.fz = S.a.fz;
    a.ux = S.a.ux;
    a.uy = S.a.uy;
    a.uz = S.a.uz;
    a.rho = c.rho[c.cur];
    a.rho_s = c.rho_scale;
    a.unit = c.rho_scale * 4294967296.0;
    a.D = c.D;
    a.r0 = c.r0;
    a.dx = c.cfg.dx;
    a.kick = c.dt / (S.mass * kC);
    a.cs0 = kC * c.dt / c.cfg.dx;
    a.lam_pos = lam_pos;
    a.lam_u = lam_u;
    a.lam_nodes = lam_nodes;
    a.grads = grads;
    return a;
}

static int agrid(const Ctx& c, int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)c.nsm * 8) g = (int64_t)c.nsm * 8;
    return g < 1 ? 1 : (int)g;
}

void launch_adjoint_seed(Ctx& c, double kin, const double* w_nodes, double* lam_pos, double* lam_u, double* lam_nodes,
                         double* r0_out, cudaStream_t st)
{
    AdjArgs a = make_adj(c, lam_pos, lam_u, lam_nodes, nullptr);
    const int64_t nn = (int64_t)c.nn;
    k_adjoint_seed<<<agrid(c, a.n > nn ? a.n : nn), 256, 0, st>>>(a, kin * c.w * c.sp[0].mass * kC * kC, w_nodes, nn,
                                                                   r0_out);
    // the final node density's dependence on the positions
    cudaMemcpyAsync(lam_nodes, w_nodes, sizeof(double) * c.nn, cudaMemcpyDeviceToDevice, st);
    k_adjoint_b<<<agrid(c, a.n), 256, 0, st>>>(a);
}

void launch_adjoint_step(Ctx& c, double* lam_pos, double* lam_u, double* lam_nodes, double* grads, cudaStream_t st)
{
    AdjArgs a = make_adj(c, lam_pos, lam_u, lam_nodes, grads);
    cudaMemsetAsync(lam_nodes, 0, sizeof(double) * c.nn, st);
    k_adjoint_a<<<agrid(c, a.n), 256, 0, st>>>(a);
    k_adjoint_b<<<agrid(c, a.n), 256, 0, st>>>(a);
}

void launch_node_functional(Ctx& c, const double* w_nodes, double* dev_out, cudaStream_t st)
{
    cudaMemsetAsync(dev_out, 0, sizeof(double), st);
    k_node_functional<<<agrid(c, (int64_t)c.nn), 256, 0, st>>>(c.rho[c.cur], c.nx, c.nz, c.rho_scale, w_nodes,
                                                                (int64_t)c.nn, dev_out);
}


// ==============================================================================================
// Part 2: the full cycle (ions, electrons, Yee fields, laser antenna). Forward step t:
//   n^ = dens(ions); per particle: E, B gathered (staggered bilinear), pair force (ions), Boris,
//   x' = x + c dt u'/(gamma' dx), walls; current j = Esirkepov(x, x', u'_y / gamma');
//   Maxwell: B += H E (half), E = M(E, B, j) with Mur walls and the antenna, B += H E (half).
// Reverse step t: Maxwell transpose (field adjoints of t+1 -> of t, current adjoints, dL/dI0),
// then per particle the transposes of the current, move, walls, Boris, gathers and pair force,
// then the density transpose. j is the scaled current dt J / eps0 with the deposition taken as
// the continuous linear shape (straight-through on the fixed point).
// Adjoint field layout (lam_F): 9 grids of (nz + 1) nx doubles: Ex Ey Ez Bx By Bz, then three
// scratch grids for the new E adjoints.
// ==============================================================================================

struct MaxAdjArgs {
    int nx, nz, k_ant;
    double hb, he, mur;        // dt / (2 dx), c^2 dt / dx, (c dt - dx) / (c dt + dx)
    double* lF;                // 9 grids
    double* lj;                // 3 grids
    const float *antc, *ants;  // antenna tables (amplitude * cos / sin of the phase)
    AntennaParams ap;          // coef = 2 c dt / dx (per unit E0)
    long long step;
    double dE0_dI0;
    double* grads;             // grads[2] += dL/dI0
};

__device__ __forceinline__ double lF_at(const MaxAdjArgs& a, int f, int i, int k)
{
    return a.lF[(size_t)f * (a.nz + 1) * a.nx + (size_t)k * a.nx + i];
}

// lam_E += H^T lam_B (transpose of a B half step; lam_B unchanged), one thread per node
__global__ void k_adj_hbT(const MaxAdjArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (i >= a.nx) return;
    const int nz = a.nz, im = i == 0 ? a.nx - 1 : i - 1;
    const size_t nn = (size_t)(nz + 1) * a.nx, c = (size_t)k * a.nx + i;
    const double bx = k < nz ? lF_at(a, 3, i, k) : 0.0, bxm = k >= 1 ? lF_at(a, 3, i, k - 1) : 0.0;
    const double by = k < nz ? lF_at(a, 4, i, k) : 0.0, bym = k >= 1 ? lF_at(a, 4, i, k - 1) : 0.0;
    const double byl = k < nz ? lF_at(a, 4, im, k) : 0.0;
    const double bz = lF_at(a, 5, i, k), bzl = lF_at(a, 5, im, k);
    a.lF[c] += a.hb * (by - bym);
    a.lF[nn + c] += a.hb * (bxm - bx - bzl + bz);
    a.lF[2 * nn + c] += a.hb * (byl - by);
}

// adjoint of the new Ex / Ey of an interior row after the Mur transposes
__device__ __forceinline__ double lnE(const MaxAdjArgs& a, int f, int i, int k)
{
    if (k <= 0 || k >= a.nz) return 0.0;
    double v = lF_at(a, f, i, k);
    if (k == 1) v += a.mur * lF_at(a, f, i, 0);
    if (k == a.nz - 1) v += a.mur * lF_at(a, f, i, a.nz);
    return v;
}

// transpose of the E update: reads the new-E adjoints (grids 0-2), updates the B adjoints in place,
// writes the old-E adjoints to grids 6-8 and the current adjoints; the antenna row adds dL/dI0
__global__ void __launch_bounds__(256) k_adj_feT(const MaxAdjArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    const int nz = a.nz;
    double g = 0.0;
    if (i < a.nx) {
        const int ip = i + 1 == a.nx ? 0 : i + 1;
        const size_t nn = (size_t)(nz + 1) * a.nx, c = (size_t)k * a.nx + i;
        const double lx = lnE(a, 0, i, k), ly = lnE(a, 1, i, k);
        double ox = lx, oy = ly;
        if (k == 1) { ox += lF_at(a, 0, i, 0); oy += lF_at(a, 1, i, 0); }
        if (k == nz - 1) { ox += lF_at(a, 0, i, nz); oy += lF_at(a, 1, i, nz); }
        if (k == 0) { ox -= a.mur * lF_at(a, 0, i, 0); oy -= a.mur * lF_at(a, 1, i, 0); }
        if (k == nz) { ox -= a.mur * lF_at(a, 0, i, nz); oy -= a.mur * lF_at(a, 1, i, nz); }
        const double lez = lF_at(a, 2, i, k);
        a.lF[6 * nn + c] = ox;
        a.lF[7 * nn + c] = oy;
        a.lF[8 * nn + c] = lez;
        double* lBx = a.lF + 3 * nn;
        double* lBy = a.lF + 4 * nn;
        double* lBz = a.lF + 5 * nn;
        lBy[c] += a.he * (lnE(a, 0, i, k + 1) - lx) + (k < nz ? a.he * (lez - lF_at(a, 2, ip, k)) : 0.0);
        lBx[c] += a.he * (ly - lnE(a, 1, i, k + 1));
        lBz[c] += a.he * (lnE(a, 1, ip, k) - ly);
        a.lj[c] = -lx;
        a.lj[nn + c] = -ly;
        a.lj[2 * nn + c] = k < nz ? -lez : 0.0;
        if (k == a.k_ant && a.ap.on) {
            const double tau = ((double)a.step + 0.5) * a.ap.dt - a.ap.t_ant;
            const double env = exp(-2.0 * 0.6931471805599453 * tau * tau / (a.ap.tau_fwhm * a.ap.tau_fwhm));
            const double s = a.ap.coef * env * sin(a.ap.omega * tau), co = a.ap.coef * env * cos(a.ap.omega * tau);
            g = lx * ((double)a.antc[i] * s + (double)a.ants[i] * co) * a.dE0_dI0;
        }
    }
    if (k == a.k_ant) {
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if ((threadIdx.x & 31) == 0 && g != 0.0) atomicAdd(a.grads + 2, g);
    }
}

struct FullAdjArgs {
    int nx, nz;
    unsigned nx_magic;
    int64_t n;
    const int32_t* cell;
    const float *fx, *fz, *ux, *uy, *uz;
    const float* F[6];
    const u64* rho;
    double rho_s;
    double D, r0, dx, dt;
    double q, m, sg;          // charge (C), mass (kg), charge sign of the current
    int pair;
    double cx, cy;            // scaled current per unit Esirkepov sum: x/z and y
    double* lam_pos;
    double* lam_u;
    double* lF;               // 6 grids (accumulated)
    const double* lj;         // 3 grids
    double* lam_nodes;
    double* grads;
};

__device__ __forceinline__ double hat_c(double d)
{
    const double a = fabs(d);
    return a < 1.0 ? 1.0 - a : 0.0;
}
__device__ __forceinline__ double dhat_c(double d) { return fabs(d) < 1.0 ? (d > 0.0 ? -1.0 : 1.0) : 0.0; }

// staggered bilinear gather of a Yee component at (i + sx, k + sz) and, if lv != 0, its transpose
__device__ __forceinline__ double gather_stag(const FullAdjArgs& a, int f, double x, double z, double sx, double sz,
                                              double lv, double& lx, double& lz)
{
    const int nx = a.nx, nz = a.nz;
    const double xs = x - sx;
    double zs = z - sz;
    const int rows = sz > 0 ? nz : nz + 1;
    bool clamped = false;
    if (zs < 0.0) { zs = 0.0; clamped = true; }
    if (zs > (double)(rows - 1)) { zs = (double)(rows - 1); clamped = true; }
    int i = (int)floor(xs), k = (int)floor(zs);
    double fx = xs - (double)i, fz = zs - (double)k;
    if (k >= rows - 1) { k = rows - 2; fz = 1.0; }
    const int i0 = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    const int i1 = i0 + 1 == nx ? 0 : i0 + 1;
    const float* A = a.F[f];
    const size_t r0 = (size_t)k * nx, r1 = r0 + nx;
    const double a00 = A[r0 + i0], a10 = A[r0 + i1], a01 = A[r1 + i0], a11 = A[r1 + i1];
    if (lv != 0.0) {
        double* L = a.lF + (size_t)f * (nz + 1) * nx;
        atomicAdd(L + r0 + i0, lv * (1 - fx) * (1 - fz));
        atomicAdd(L + r0 + i1, lv * fx * (1 - fz));
        atomicAdd(L + r1 + i0, lv * (1 - fx) * fz);
        atomicAdd(L + r1 + i1, lv * fx * fz);
        lx += lv * ((1 - fz) * (a10 - a00) + fz * (a11 - a01));
        if (!clamped) lz += lv * ((1 - fx) * (a01 - a00) + fx * (a11 - a10));
    }
    return (1 - fx) * (1 - fz) * a00 + fx * (1 - fz) * a10 + (1 - fx) * fz * a01 + fx * fz * a11;
}

__device__ __forceinline__ double node_n_full(const FullAdjArgs& a, int i, int k)
{
    const long long v = (long long)a.rho[(size_t)k * a.nx + i];
    return a.rho_s * (double)((k == 0 || k == a.nz) ? 2 * v : v);
}

// transpose of the continuous Esirkepov current of one particle: adds d/d(x0, z0, x1, z1, by) of
// sum lj * j into g[0..4]
__device__ void cur_T(const FullAdjArgs& a, double x0, double z0, double x1, double z1, double by, double g[5])
{
    const int nx = a.nx, nz = a.nz;
    const double bx = floor(fmin(x0, x1)), bz = floor(fmin(z0, z1));
    const int ib = (int)bx, kb = (int)bz;
    double S0x[3], S1x[3], S0z[3], S1z[3];
    double Lx[3][3], Ly[3][3], Lz[3][3];
    const size_t nn = (size_t)(nz + 1) * nx;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        S0x[q] = hat_c(x0 - (bx + q));
        S1x[q] = hat_c(x1 - (bx + q));
        S0z[q] = hat_c(z0 - (bz + q));
        S1z[q] = hat_c(z1 - (bz + q));
    }
#pragma unroll
    for (int ia = 0; ia < 3; ia++) {
        int ii = ib + ia;
        ii = ii < 0 ? ii + nx : (ii >= nx ? ii - nx : ii);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const int l = kb + b;
            const bool ok = l >= 0 && l <= nz;
            const size_t c = (size_t)l * nx + ii;
            Lx[ia][b] = ok ? a.lj[c] : 0.0;
            Ly[ia][b] = ok ? a.lj[nn + c] : 0.0;
            Lz[ia][b] = ok ? a.lj[2 * nn + c] : 0.0;
        }
    }
    const double cx = a.sg * a.cx, cy = a.sg * a.cy;
    double dS0x[3] = {0, 0, 0}, dS1x[3] = {0, 0, 0}, dS0z[3] = {0, 0, 0}, dS1z[3] = {0, 0, 0};
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const double Rx1 = Lx[1][b], Rx0 = Lx[0][b] + Lx[1][b], zsum = S0z[b] + S1z[b];
        dS1x[0] -= cx * zsum * Rx0; dS0x[0] += cx * zsum * Rx0;
        dS1x[1] -= cx * zsum * Rx1; dS0x[1] += cx * zsum * Rx1;
        const double zz = -cx * ((S1x[0] - S0x[0]) * Rx0 + (S1x[1] - S0x[1]) * Rx1);
        dS0z[b] += zz; dS1z[b] += zz;
    }
#pragma unroll
    for (int ia = 0; ia < 3; ia++) {
        const double Rz1 = Lz[ia][1], Rz0 = Lz[ia][0] + Lz[ia][1], xsum = S0x[ia] + S1x[ia];
        dS1z[0] -= cx * xsum * Rz0; dS0z[0] += cx * xsum * Rz0;
        dS1z[1] -= cx * xsum * Rz1; dS0z[1] += cx * xsum * Rz1;
        const double xx = -cx * ((S1z[0] - S0z[0]) * Rz0 + (S1z[1] - S0z[1]) * Rz1);
        dS0x[ia] += xx; dS1x[ia] += xx;
    }
    double gby = 0.0;
#pragma unroll
    for (int ia = 0; ia < 3; ia++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const double L = Ly[ia][b] * cy;
            gby += L * (2 * S0x[ia] * S0z[b] + S1x[ia] * S0z[b] + S0x[ia] * S1z[b] + 2 * S1x[ia] * S1z[b]);
            dS0x[ia] += by * L * (2 * S0z[b] + S1z[b]);
            dS1x[ia] += by * L * (S0z[b] + 2 * S1z[b]);
            dS0z[b] += by * L * (2 * S0x[ia] + S1x[ia]);
            dS1z[b] += by * L * (S0x[ia] + 2 * S1x[ia]);
        }
#pragma unroll
    for (int q = 0; q < 3; q++) {
        g[0] += dS0x[q] * dhat_c(x0 - (bx + q));
        g[1] += dS0z[q] * dhat_c(z0 - (bz + q));
        g[2] += dS1x[q] * dhat_c(x1 - (bx + q));
        g[3] += dS1z[q] * dhat_c(z1 - (bz + q));
    }
    g[4] += gby;
}

__device__ __constant__ double c_stag[6][2] = {{0.5, 0.0}, {0.0, 0.0}, {0.0, 0.5}, {0.0, 0.5}, {0.5, 0.5}, {0.5, 0.0}};

__global__ void __launch_bounds__(256) k_adjoint_full(const FullAdjArgs a)
{
    __shared__ double sh[256];
    double gD = 0.0, gR = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        int ci, ck;
        split2(a.cell[p], a.nx, a.nx_magic, ci, ck);
        const double x = (double)ci + (double)a.fx[p], z = (double)ck + (double)a.fz[p];
        // ---- forward recompute (FP64) ----
        double E[3], B[3], dummy = 0.0;
#pragma unroll
        for (int f = 0; f < 6; f++) {
            const double v = gather_stag(a, f, x, z, c_stag[f][0], c_stag[f][1], 0.0, dummy, dummy);
            if (f < 3) E[f] = v; else B[f - 3] = v;
        }
        double Fp[3] = {0.0, 0.0, 0.0};
        double n = 0, qx = 0, qz = 0, gxz = 0, dxn = 0, dxq = 0, dxr = 0, dzn = 0, dzq = 0, dzr = 0, pfx = 0, pfz = 0;
        int pi = 0, pk = 0;
        if (a.pair) {
            double fx = a.fx[p], fz = a.fz[p];
            pi = ci; pk = ck;
            if (pk >= a.nz) { pk = a.nz - 1; fz = 1.0; }
            const int i1 = pi + 1 == a.nx ? 0 : pi + 1;
            const double n00 = node_n_full(a, pi, pk), n10 = node_n_full(a, i1, pk);
            const double n01 = node_n_full(a, pi, pk + 1), n11 = node_n_full(a, i1, pk + 1);
            n = (1 - fx) * (1 - fz) * n00 + fx * (1 - fz) * n10 + (1 - fx) * fz * n01 + fx * fz * n11;
            qx = (1 - fz) * (n10 - n00) + fz * (n11 - n01);
            qz = (1 - fx) * (n01 - n00) + fx * (n11 - n10);
            gxz = n11 - n01 - n10 + n00;
            Fp[0] = axis_force_d(n, qx, a.D, a.r0, a.dx, dxn, dxq, dxr);
            Fp[2] = axis_force_d(n, qz, a.D, a.r0, a.dx, dzn, dzq, dzr);
            pfx = fx; pfz = fz;
        }
        const double eps = a.q * a.dt / (2.0 * a.m * kC), fk = a.dt / (2.0 * a.m * kC);
        double um[3], t[3], sv[3], upr[3], uf[3];
        const double u0[3] = {(double)a.ux[p], (double)a.uy[p], (double)a.uz[p]};
#pragma unroll
        for (int d = 0; d < 3; d++) um[d] = u0[d] + eps * E[d] + fk * Fp[d];
        const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        const double tfac = a.q * a.dt / (2.0 * a.m * gm);
#pragma unroll
        for (int d = 0; d < 3; d++) t[d] = tfac * B[d];
        const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
#pragma unroll
        for (int d = 0; d < 3; d++) sv[d] = 2.0 * t[d] / (1.0 + t2);
        upr[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
        upr[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
        upr[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
        uf[0] = um[0] + (upr[1] * sv[2] - upr[2] * sv[1]) + eps * E[0] + fk * Fp[0];
        uf[1] = um[1] + (upr[2] * sv[0] - upr[0] * sv[2]) + eps * E[1] + fk * Fp[1];
        uf[2] = um[2] + (upr[0] * sv[1] - upr[1] * sv[0]) + eps * E[2] + fk * Fp[2];
        const double g = sqrt(1.0 + uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
        const double cs = kC * a.dt / (g * a.dx);
        const double xn = x + uf[0] * cs, zn = z + uf[2] * cs;
        double z1 = zn, ufz_fin = uf[2];
        bool refl = false;
        if (zn < 0.0) { z1 = -zn; ufz_fin = -uf[2]; refl = true; }
        if (zn >= (double)a.nz) { z1 = 2.0 * a.nz - zn; ufz_fin = -uf[2]; refl = true; }
        const double by = uf[1] / g;
        // ---- reverse ----
        double lx1 = a.lam_pos[2 * p], lz1 = a.lam_pos[2 * p + 1];
        double luf[3] = {a.lam_u[3 * p], a.lam_u[3 * p + 1], a.lam_u[3 * p + 2]};
        double lx0 = 0.0, lz0 = 0.0;
        if (a.sg != 0.0) {
            double g5[5] = {0, 0, 0, 0, 0};
            cur_T(a, x, z, xn, z1, by, g5);
            lx0 += g5[0]; lz0 += g5[1]; lx1 += g5[2]; lz1 += g5[3];
            const double ufin[3] = {uf[0], uf[1], ufz_fin};
            const double g3 = g * g * g;
#pragma unroll
            for (int d = 0; d < 3; d++) luf[d] += g5[4] * ((d == 1 ? 1.0 / g : 0.0) - ufin[1] * ufin[d] / g3);
        }
        double lzn = lz1;
        if (refl) { lzn = -lz1; luf[2] = -luf[2]; }
        const double udl = (uf[0] * lx1 + uf[2] * lzn) / (g * g);
        double lu[3];
        lu[0] = luf[0] + cs * (lx1 - uf[0] * udl);
        lu[1] = luf[1] + cs * (0.0 - uf[1] * udl);
        lu[2] = luf[2] + cs * (lzn - uf[2] * udl);
        lx0 += lx1;
        lz0 += lzn;
        // Boris transpose
        double la[3], lum[3], lupr[3], lsv[3], lt[3];
#pragma unroll
        for (int d = 0; d < 3; d++) { la[d] = lu[d]; lum[d] = lu[d]; }
        lupr[0] = sv[1] * lu[2] - sv[2] * lu[1];
        lupr[1] = sv[2] * lu[0] - sv[0] * lu[2];
        lupr[2] = sv[0] * lu[1] - sv[1] * lu[0];
        lsv[0] = lu[1] * upr[2] - lu[2] * upr[1];
        lsv[1] = lu[2] * upr[0] - lu[0] * upr[2];
        lsv[2] = lu[0] * upr[1] - lu[1] * upr[0];
        lum[0] += lupr[0] + (t[1] * lupr[2] - t[2] * lupr[1]);
        lum[1] += lupr[1] + (t[2] * lupr[0] - t[0] * lupr[2]);
        lum[2] += lupr[2] + (t[0] * lupr[1] - t[1] * lupr[0]);
        lt[0] = lupr[1] * um[2] - lupr[2] * um[1];
        lt[1] = lupr[2] * um[0] - lupr[0] * um[2];
        lt[2] = lupr[0] * um[1] - lupr[1] * um[0];
        const double tl = t[0] * lsv[0] + t[1] * lsv[1] + t[2] * lsv[2], d1 = 1.0 + t2;
#pragma unroll
        for (int d = 0; d < 3; d++) lt[d] += 2.0 * lsv[d] / d1 - 4.0 * tl * t[d] / (d1 * d1);
        double lB[3], ltf = 0.0;
#pragma unroll
        for (int d = 0; d < 3; d++) { lB[d] = tfac * lt[d]; ltf += B[d] * lt[d]; }
        const double lgm = -tfac / gm * ltf;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            lum[d] += lgm * um[d] / gm;
            la[d] += lum[d];
        }
        a.lam_u[3 * p] = lum[0];
        a.lam_u[3 * p + 1] = lum[1];
        a.lam_u[3 * p + 2] = lum[2];
        // field gathers
#pragma unroll
        for (int f = 0; f < 6; f++) {
            const double lv = f < 3 ? eps * la[f] : lB[f - 3];
            gather_stag(a, f, x, z, c_stag[f][0], c_stag[f][1], lv, lx0, lz0);
        }
        // pair force (ions)
        if (a.pair) {
            const double lFx = fk * la[0], lFz = fk * la[2];
            gD += (lFx * Fp[0] + lFz * Fp[2]) / a.D;
            gR += lFx * (dxr + dxn * 3.0 * n / a.r0 + dxq * 3.0 * qx / a.r0) +
                  lFz * (dzr + dzn * 3.0 * n / a.r0 + dzq * 3.0 * qz / a.r0);
            const double ln = lFx * dxn + lFz * dzn, lqx = lFx * dxq, lqz = lFz * dzq;
            lx0 += ln * qx + lqz * gxz;
            lz0 += ln * qz + lqx * gxz;
            const int i1 = pi + 1 == a.nx ? 0 : pi + 1;
            double* L0 = a.lam_nodes + (size_t)pk * a.nx;
            double* L1 = L0 + a.nx;
            const double fx = pfx, fz = pfz;
            atomicAdd(L0 + pi, ln * (1 - fx) * (1 - fz) - lqx * (1 - fz) - lqz * (1 - fx));
            atomicAdd(L0 + i1, ln * fx * (1 - fz) + lqx * (1 - fz) - lqz * fx);
            atomicAdd(L1 + pi, ln * (1 - fx) * fz - lqx * fz + lqz * (1 - fx));
            atomicAdd(L1 + i1, ln * fx * fz + lqx * fz + lqz * fx);
        }
        a.lam_pos[2 * p] = lx0;
        a.lam_pos[2 * p + 1] = lz0;
    }
    if (a.pair) {
        const double sD = block_sum_d(gD, sh), sR = block_sum_d(gR, sh);
        if (threadIdx.x == 0) {
            atomicAdd(a.grads, sD);
            atomicAdd(a.grads + 1, sR);
        }
    }
}

__global__ void k_adjoint_seed_u(int64_t n, const float* ux, const float* uy, const float* uz, double kin_mc2w,
                                 double* lam_pos, double* lam_u)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double x = ux[p], y = uy[p], z = uz[p];
        const double g = sqrt(1.0 + x * x + y * y + z * z);
        lam_u[3 * p] = kin_mc2w * x / g;
        lam_u[3 * p + 1] = kin_mc2w * y / g;
        lam_u[3 * p + 2] = kin_mc2w * z / g;
        lam_pos[2 * p] = 0.0;
        lam_pos[2 * p + 1] = 0.0;
    }
}

static FullAdjArgs make_full_adj(Ctx& c, int s, double* const* lam_pos, double* const* lam_u, double* lam_nodes,
                                 double* lF, const double* lj, double* grads)
{
    FullAdjArgs a;
    a.nx = c.nx;
    a.nz = c.nz;
    a.nx_magic = (unsigned)(4294967296ULL / (unsigned long long)c.nx);
    const Species& S = c.sp[s];
    a.n = S.n;
    a.cell = S.a.cell;
    a.fx = S.a.fx;
    a.fz = S.a.fz;
    a.ux = S.a.ux;
    a.uy = S.a.uy;
    a.uz = S.a.uz;
    for (int q = 0; q < 6; q++) a.F[q] = c.F[q];
    a.rho = c.rho[c.cur];
    a.rho_s = c.rho_scale;
    a.D = c.D;
    a.r0 = c.r0;
    a.dx = c.cfg.dx;
    a.dt = c.dt;
    a.q = s == 0 ? c.cfg.ion_charge * kQe : -kQe;
    a.m = S.mass;
    a.sg = (double)S.jsign;
    a.pair = S.pair;
    a.cx = kQe * c.w / (2.0 * c.cfg.dx * kEps0);
    a.cy = kQe * c.w * kC * c.dt / (6.0 * c.cfg.dx * c.cfg.dx * kEps0);
    a.lam_pos = lam_pos[s];
    a.lam_u = lam_u[s];
    a.lF = lF;
    a.lj = lj;
    a.lam_nodes = lam_nodes;
    a.grads = grads;
    return a;
}

void launch_adjoint_seed_full(Ctx& c, double kin, const double* w_nodes, double* const* lam_pos, double* const* lam_u,
                              double* lam_nodes, double* lF, double* lj, double* r0_out, cudaStream_t st)
{
    const size_t nn = c.nn;
    cudaMemsetAsync(lF, 0, sizeof(double) * 9 * nn, st);
    cudaMemsetAsync(lj, 0, sizeof(double) * 3 * nn, st);
    for (int s = 0; s < c.nsp; s++) {
        const Species& S = c.sp[s];
        k_adjoint_seed_u<<<agrid(c, S.n), 256, 0, st>>>(S.n, S.a.ux, S.a.uy, S.a.uz, kin * c.w * S.mass * kC * kC,
                                                         lam_pos[s], lam_u[s]);
    }
    if (c.sp[0].pair) {
        // the pair species' density: r0 term and the transpose of the final deposition
        AdjArgs a = make_adj(c, lam_pos[0], lam_u[0], lam_nodes, nullptr);
        AdjArgs nodes_only = a;
        nodes_only.n = 0;                                  // momenta seeded above
        k_adjoint_seed<<<agrid(c, (int64_t)nn), 256, 0, st>>>(nodes_only, 0.0, w_nodes, (int64_t)nn, r0_out);
        cudaMemcpyAsync(lam_nodes, w_nodes, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st);
        k_adjoint_b<<<agrid(c, a.n), 256, 0, st>>>(a);
    }
}

void launch_adjoint_step_full(Ctx& c, double* const* lam_pos, double* const* lam_u, double* lam_nodes, double* lF,
                              double* lj, double* grads, cudaStream_t st)
{
    const size_t nn = c.nn;
    MaxAdjArgs m;
    m.nx = c.nx;
    m.nz = c.nz;
    m.k_ant = c.k_ant;
    m.hb = 0.5 * c.dt / c.cfg.dx;
    m.he = kC * kC * c.dt / c.cfg.dx;
    const double cdt = kC * c.dt;
    m.mur = (cdt - c.cfg.dx) / (cdt + c.cfg.dx);
    m.lF = lF;
    m.lj = lj;
    m.antc = c.ant_c;
    m.ants = c.ant_s;
    m.ap = make_antenna_params(c);
    m.ap.coef = 2.0 * (kC * c.dt / c.cfg.dx);            // per unit E0
    m.step = (long long)c.step;
    m.dE0_dI0 = c.cfg.I0 > 0 ? c.E0 / (2.0 * c.cfg.I0) : 0.0;
    m.grads = grads;
    const dim3 block(256), grid((c.nx + 255) / 256, c.nz + 1);
    k_adj_hbT<<<grid, block, 0, st>>>(m);
    k_adj_feT<<<grid, block, 0, st>>>(m);
    cudaMemcpyAsync(lF, lF + 6 * nn, sizeof(double) * 3 * nn, cudaMemcpyDeviceToDevice, st);
    k_adj_hbT<<<grid, block, 0, st>>>(m);
    if (c.sp[0].pair) cudaMemsetAsync(lam_nodes, 0, sizeof(double) * nn, st);
    for (int s = 0; s < c.nsp; s++) {
        FullAdjArgs a = make_full_adj(c, s, lam_pos, lam_u, lam_nodes, lF, lj, grads);
        if (a.n > 0) k_adjoint_full<<<agrid(c, a.n), 256, 0, st>>>(a);
    }
    if (c.sp[0].pair) {
        AdjArgs b = make_adj(c, lam_pos[0], lam_u[0], lam_nodes, grads);
        k_adjoint_b<<<agrid(c, b.n), 256, 0, st>>>(b);
    }
}

}  // namespace gbpic
