// Reverse-mode (adjoint) kernels of the atomic-transport stage in 2D: neutral atoms, pair force
// only (paper: the transport simulation evolves the target with the pair potential). They give
// gradients of a loss of the final state with respect to the pair-potential parameters D and r0
// (r0 sets Eq. (3)'s equilibrium distance, the r0/dx of Eq. (1), and the density unit
// n0 = r0^-3).
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

}  // namespace gbpic
