// Reverse-mode (adjoint) kernels of the 2D cycle, for gradients of a loss of the final state with
// respect to the pair-potential parameters D and r0 (r0 sets Eq. (3)'s equilibrium distance, the
// r0/dx of Eq. (1), and the density unit n0 = r0^-3) and, with fields, the laser peak intensity.
//
// Precision: the per-particle transposes run in FP32 (the precision of the forward push) and
// scatter onto the nodes with FP32 atomics; the field adjoints are held and transposed through
// the Yee step in FP64 on the nodes (the particle scatter is folded in once per step), and the
// parameter derivatives are summed in FP64. The deposition is
// differentiated as the continuous linear shape (straight-through on the fixed point). Node
// density differences are taken exactly in integers before scaling.
//
// Part 1: the atomic-transport stage (neutral atoms, pair force only; paper: the transport
// simulation evolves the target with the pair potential).
// Forward step (per atom): node density n(x) -> gather (n, dn/dxi, dn/dzeta) -> force F(n, q) of
// Eqs. (1)-(3) -> u += F dt / (m c) -> x += c dt u / (gamma dx) -> wall mirror.
// One reverse step (kernels A and B) maps the adjoints of (x^(t+1), u^(t+1)) to those of
// (x^t, u^t) and accumulates the parameter gradients:
//   A: per atom -- transpose of the position update and of the kick, force derivatives, the
//      gather's position derivatives, and the gather's transpose onto the nodes;
//   B: per atom -- transpose of the deposition: the node adjoints' interpolated gradient.
#include "pic_device.cuh"

namespace gbpic {

// ---- pair force of one axis and its derivatives, Eqs. (1)-(3) -----------------------------------
// With c = n^(1/3) (n in units of n0) and h = g/2 = -(1/6)(r0/dx) n^(-4/3) q, the neighbours sit at
// 1/(c(1-h)) and 1/(c(1+h)) (units of r0), and
//   F = (D/r0) [U'(a) - U'(b)] = 12 (D/r0) c^7 (c^6 P13(h) - P7(h)),
//   P_m(h) = (1+h)^m - (1-h)^m (odd polynomials, written out), which has no cancellation between
// the two neighbours' terms; for |h| >= 1 a neighbour is at infinity and the terms are separate.
struct PairD {
    float F, dn, dq, dr0;   // force (N) and dF/dn, dF/dq (fixed n, q), dF/dr0 (fixed n, q)
};

__device__ __forceinline__ PairD pair_axis_d(float n, float q, float r0_dx, float fu, float inv_r0)
{
    PairD o = {0.0f, 0.0f, 0.0f, 0.0f};
    if (!(n > 0.0f)) return o;
    const float c = cbrtf(n);
    const float inc = 1.0f / (n * c);                       // n^(-4/3)
    const float h = -(1.0f / 6.0f) * r0_dx * q * inc;
    const float c2 = c * c, c6 = c2 * c2 * c2, c7 = c6 * c;
    float F, dFdc, dFdh;
    if (fabsf(h) < 1.0f) {
        const float h2 = h * h;
        const float P7 = 2.0f * h * (7.0f + h2 * (35.0f + h2 * (21.0f + h2)));
        const float P13 = 2.0f * h * (13.0f + h2 * (286.0f + h2 * (1287.0f + h2 * (1716.0f + h2 * (715.0f + h2 * (78.0f + h2))))));
        const float D7 = 14.0f * (1.0f + h2 * (15.0f + h2 * (15.0f + h2)));
        const float D13 = 26.0f * (1.0f + h2 * (66.0f + h2 * (495.0f + h2 * (924.0f + h2 * (495.0f + h2 * (66.0f + h2))))));
        F = 12.0f * fu * c7 * (c6 * P13 - P7);
        dFdc = 12.0f * fu * c6 * (13.0f * c6 * P13 - 7.0f * P7);
        dFdh = 12.0f * fu * c7 * (c6 * D13 - D7);
    } else {
        F = dFdc = dFdh = 0.0f;
        if (1.0f - h > 0.0f) {
            const float ia = c * (1.0f - h), i2 = ia * ia, i6 = i2 * i2 * i2;
            const float d = 12.0f * fu * i6 * (7.0f - 13.0f * i6);    // (D/r0) dU'(a)/d(1/a)
            F += 12.0f * fu * i6 * ia * (1.0f - i6);
            dFdc += d * (1.0f - h);
            dFdh -= d * c;
        }
        if (1.0f + h > 0.0f) {
            const float ib = c * (1.0f + h), i2 = ib * ib, i6 = i2 * i2 * i2;
            const float d = 12.0f * fu * i6 * (7.0f - 13.0f * i6);
            F -= 12.0f * fu * i6 * ib * (1.0f - i6);
            dFdc -= d * (1.0f + h);
            dFdh -= d * c;
        }
    }
    const float inv_n = 1.0f / n;
    o.F = F;
    o.dn = dFdc * c * (1.0f / 3.0f) * inv_n - dFdh * (4.0f / 3.0f) * h * inv_n;
    o.dq = -dFdh * (1.0f / 6.0f) * r0_dx * inc;
    o.dr0 = (dFdh * h - F) * inv_r0;
    return o;
}

// the pair-species density around a particle: bilinear value, exact edge differences, and the
// pieces the transpose needs
struct DensAt {
    float n, qx, qz, gxz, fx, fz;
    int i, i1, k;
};

// int64 -> FP32 through two 32-bit conversions: the 64-bit conversion runs on GB300's slow FP64 pipe
// (9 per particle here); the result differs from the correctly rounded one by at most one rounding
__device__ __forceinline__ float i64f(long long v)
{
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)v;
    return fmaf((float)hi, 4294967296.0f, (float)lo);
}

__device__ __forceinline__ long long node_sum(const u64* rho, int nx, int nz, int i, int k)
{
    const long long v = (long long)rho[(size_t)k * nx + i];
    return (k == 0 || k == nz) ? 2 * v : v;
}

__device__ __forceinline__ DensAt dens_at(const u64* rho, float rho_s, int nx, int nz, int ci, int ck, float fx,
                                          float fz)
{
    DensAt d;
    if (ck >= nz) { ck = nz - 1; fz = 1.0f; }
    d.i = ci;
    d.i1 = ci + 1 == nx ? 0 : ci + 1;
    d.k = ck;
    d.fx = fx;
    d.fz = fz;
    const long long N00 = node_sum(rho, nx, nz, d.i, ck), N10 = node_sum(rho, nx, nz, d.i1, ck);
    const long long N01 = node_sum(rho, nx, nz, d.i, ck + 1), N11 = node_sum(rho, nx, nz, d.i1, ck + 1);
    const float n00 = rho_s * i64f(N00), n10 = rho_s * i64f(N10), n01 = rho_s * i64f(N01), n11 = rho_s * i64f(N11);
    d.n = (1 - fx) * (1 - fz) * n00 + fx * (1 - fz) * n10 + (1 - fx) * fz * n01 + fx * fz * n11;
    const float ex0 = rho_s * i64f(N10 - N00), ex1 = rho_s * i64f(N11 - N01);
    const float ez0 = rho_s * i64f(N01 - N00), ez1 = rho_s * i64f(N11 - N10);
    d.qx = (1 - fz) * ex0 + fz * ex1;
    d.qz = (1 - fx) * ez0 + fx * ez1;
    d.gxz = rho_s * i64f(N11 - N01 - N10 + N00);
    return d;
}

// transpose of the pair force given the adjoints of (Fx, Fz): position adjoints (added to lx, lz),
// node adjoints (FP64 atomics), and the D, r0 derivative terms (gFF += lF . F, gR += dL/dr0 part)
__device__ __forceinline__ void pair_T(const DensAt& d, const PairD& px, const PairD& pz, float lFx, float lFz,
                                       float inv_r0, int nx, float* lam_nodes, float& lx, float& lz, double& gFF,
                                       double& gR)
{
    gFF += (double)(lFx * px.F + lFz * pz.F);
    gR += (double)(lFx * (px.dr0 + 3.0f * inv_r0 * (px.dn * d.n + px.dq * d.qx)) +
                   lFz * (pz.dr0 + 3.0f * inv_r0 * (pz.dn * d.n + pz.dq * d.qz)));
    const float ln = lFx * px.dn + lFz * pz.dn, lqx = lFx * px.dq, lqz = lFz * pz.dq;
    lx += ln * d.qx + lqz * d.gxz;
    lz += ln * d.qz + lqx * d.gxz;
    const float fx = d.fx, fz = d.fz;
    float* L0 = lam_nodes + (size_t)d.k * nx;
    float* L1 = L0 + nx;
    atomicAdd(L0 + d.i, ln * (1 - fx) * (1 - fz) - lqx * (1 - fz) - lqz * (1 - fx));
    atomicAdd(L0 + d.i1, ln * fx * (1 - fz) + lqx * (1 - fz) - lqz * fx);
    atomicAdd(L1 + d.i, ln * (1 - fx) * fz - lqx * fz + lqz * (1 - fx));
    atomicAdd(L1 + d.i1, ln * fx * fz + lqx * fz + lqz * fx);
}

__device__ __forceinline__ void split2(int cell, int nx, unsigned magic, int& i, int& k)
{
    unsigned q = __umulhi((unsigned)cell, magic);
    int r = cell - (int)q * nx;
    if (r >= nx) { q++; r -= nx; }
    k = (int)q;
    i = r;
}

// Particle of this thread in chunk `ch` (blocks of 256 threads take chunks of 256 consecutive
// records). The cell sort's storage layout already gives the 32 consecutive records of a warp 32
// different cells (runs of the cell order side by side), so a warp's node atomics rarely share an
// address while its loads stay coalesced.
__device__ __forceinline__ int64_t spread_index(int64_t ch) { return ch * 256 + (int64_t)threadIdx.x; }

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

struct AdjArgs {
    int nx, nz;
    unsigned nx_magic;
    int64_t n;
    const int32_t* cell;
    const float *fx, *fz, *ux, *uy, *uz;
    const u64* rho;        // fixed-point node sums at the current positions
    double rho_s;          // node sum -> n / n0
    double unit;           // one particle's full weight on a node, in units of n0 (rho_s * 2^32)
    double D, r0, dx, kick, cs0;   // kick = dt / (m c); cs0 = c dt / dx
    float* lam_pos;        // 2 n: (x, z) adjoints
    float* lam_u;          // 3 n
    float* lam_nodes;      // (nz + 1) nx node adjoints (units 1 / n0)
    double* grads;         // 3: dL/dD, dL/dr0, dL/dI0
};

__global__ void __launch_bounds__(256) k_adjoint_a(const AdjArgs a)
{
    __shared__ double sh[256];
    double gFF = 0.0, gR = 0.0;
    const float r0_dx = (float)(a.r0 / a.dx), fu = (float)(a.D / a.r0), inv_r0 = (float)(1.0 / a.r0);
    const float rho_s = (float)a.rho_s, kick = (float)a.kick, cs0 = (float)a.cs0;
    for (int64_t ch = blockIdx.x; ch * 256 < a.n; ch += gridDim.x) {
        const int64_t p = spread_index(ch);
        if (p >= a.n) continue;
        int ci, ck;
        split2(a.cell[p], a.nx, a.nx_magic, ci, ck);
        const float fx = a.fx[p], fz = a.fz[p];
        const DensAt d = dens_at(a.rho, rho_s, a.nx, a.nz, ci, ck, fx, fz);
        const PairD px = pair_axis_d(d.n, d.qx, r0_dx, fu, inv_r0), pz = pair_axis_d(d.n, d.qz, r0_dx, fu, inv_r0);
        // forward quantities of this step: kicked momentum (before the wall mirror), move
        const float ux = a.ux[p] + kick * px.F, uy = a.uy[p], uz = a.uz[p] + kick * pz.F;
        const float g = sqrtf(1.0f + ux * ux + uy * uy + uz * uz), cs = cs0 / g;
        const float zl = fz + uz * cs;
        const bool refl = (ck == 0 && zl < 0.0f) || (ck == a.nz - 1 && zl >= 1.0f);
        float lpx = a.lam_pos[2 * p], lpz = a.lam_pos[2 * p + 1];
        float lux = a.lam_u[3 * p], luy = a.lam_u[3 * p + 1], luz = a.lam_u[3 * p + 2];
        if (refl) { lpz = -lpz; luz = -luz; }
        // position update x' = x + cs u: dx'/du = cs (I - u u^T / gamma^2)
        const float udl = (ux * lpx + uz * lpz) / (g * g);
        lux += cs * (lpx - ux * udl);
        luy += cs * (0.0f - uy * udl);
        luz += cs * (lpz - uz * udl);
        // kick u' = u + kick F
        float lx = lpx, lz = lpz;
        pair_T(d, px, pz, kick * lux, kick * luz, inv_r0, a.nx, a.lam_nodes, lx, lz, gFF, gR);
        a.lam_pos[2 * p] = lx;
        a.lam_pos[2 * p + 1] = lz;
        a.lam_u[3 * p] = lux;
        a.lam_u[3 * p + 1] = luy;
        a.lam_u[3 * p + 2] = luz;
    }
    const double sD = block_sum_d(gFF, sh), sR = block_sum_d(gR, sh);
    if (threadIdx.x == 0) {
        atomicAdd(a.grads, sD / a.D);
        atomicAdd(a.grads + 1, sR);
    }
}

// lam_pos += d/dx of sum_nodes lam_nodes * n^(nodes) (transpose of the deposition)
__global__ void __launch_bounds__(256) k_adjoint_b(const AdjArgs a)
{
    for (int64_t ch = blockIdx.x; ch * 256 < a.n; ch += gridDim.x) {
        const int64_t p = spread_index(ch);
        if (p >= a.n) continue;
        int i, k;
        split2(a.cell[p], a.nx, a.nx_magic, i, k);
        float fx = a.fx[p], fz = a.fz[p];
        if (k >= a.nz) { k = a.nz - 1; fz = 1.0f; }
        const int i1 = i + 1 == a.nx ? 0 : i + 1;
        const float m0 = k == 0 ? 2.0f : 1.0f, m1 = k + 1 == a.nz ? 2.0f : 1.0f;
        const float* L0 = a.lam_nodes + (size_t)k * a.nx;
        const float* L1 = L0 + a.nx;
        const float l00 = m0 * L0[i], l10 = m0 * L0[i1], l01 = m1 * L1[i], l11 = m1 * L1[i1];
        const float u = (float)a.unit;
        const float ex0 = l10 - l00, ex1 = l11 - l01, ez0 = l01 - l00, ez1 = l11 - l10;
        a.lam_pos[2 * p] += u * ((1 - fz) * ex0 + fz * ex1);
        a.lam_pos[2 * p + 1] += u * ((1 - fx) * ez0 + fx * ez1);
    }
}

// seed: lam_u = kin * w m c^2 u / gamma (lam_pos = 0); sum of lam_nodes * 3 n / r0 (the density
// unit's r0 dependence)
__global__ void __launch_bounds__(256) k_adjoint_seed(const AdjArgs a, double kin_mc2w, const double* w_nodes,
                                                      int64_t nn, double* r0_out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    const float kw = (float)kin_mc2w;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        const float ux = a.ux[p], uy = a.uy[p], uz = a.uz[p];
        const float ig = kw / sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        a.lam_u[3 * p] = ig * ux;
        a.lam_u[3 * p + 1] = ig * uy;
        a.lam_u[3 * p + 2] = ig * uz;
        a.lam_pos[2 * p] = 0.0f;
        a.lam_pos[2 * p + 1] = 0.0f;
    }
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nn; c += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / a.nx), i = (int)(c - (int64_t)k * a.nx);
        acc += w_nodes[c] * 3.0 * a.rho_s * (double)node_sum(a.rho, a.nx, a.nz, i, k) / a.r0;
        a.lam_nodes[c] = (float)w_nodes[c];                  // the final density's node adjoints
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

static AdjArgs make_adj(Ctx& c, int s, float* lam_pos, float* lam_u, float* lam_nodes, double* grads)
{
    AdjArgs a;
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

// seed of the pair species: momenta (kin), the final density functional's position adjoints and
// its r0 term
static void seed_pair_species(Ctx& c, double kin, const double* w_nodes, float* lam_pos, float* lam_u,
                              float* lam_nodes, double* r0_out, cudaStream_t st)
{
    AdjArgs a = make_adj(c, 0, lam_pos, lam_u, lam_nodes, nullptr);
    const int64_t nn = (int64_t)c.nn;
    k_adjoint_seed<<<agrid(c, a.n > nn ? a.n : nn), 256, 0, st>>>(a, kin * c.w * c.sp[0].mass * kC * kC, w_nodes, nn,
                                                                   r0_out);
    k_adjoint_b<<<agrid(c, a.n), 256, 0, st>>>(a);
}

void launch_adjoint_seed(Ctx& c, double kin, const double* w_nodes, float* lam_pos, float* lam_u, float* lam_nodes,
                         double* r0_out, cudaStream_t st)
{
    seed_pair_species(c, kin, w_nodes, lam_pos, lam_u, lam_nodes, r0_out, st);
}

void launch_adjoint_step(Ctx& c, float* lam_pos, float* lam_u, float* lam_nodes, double* grads, cudaStream_t st)
{
    AdjArgs a = make_adj(c, 0, lam_pos, lam_u, lam_nodes, grads);
    cudaMemsetAsync(lam_nodes, 0, sizeof(float) * c.nn, st);
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
// then the density transpose. j is the scaled current dt J / eps0.
// Adjoint field layout (lam_F): 9 grids of (nz + 1) nx doubles: Ex Ey Ez Bx By Bz, then three
// scratch grids: the new E adjoints during the Maxwell transpose, then (as six float grids) the
// particles' FP32 scatter onto the field nodes, folded into the first six grids after the particle
// kernels. Current adjoints (lam_j): 3 grids of floats.
// ==============================================================================================

struct MaxAdjArgs {
    int nx, nz, k_ant;
    double hb, he, mur;        // dt / (2 dx), c^2 dt / dx, (c dt - dx) / (c dt + dx)
    double* lF;                // 9 grids
    float* lj;                 // 3 grids
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
        a.lj[c] = (float)-lx;
        a.lj[nn + c] = (float)-ly;
        a.lj[2 * nn + c] = k < nz ? (float)-lez : 0.0f;
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
    float rho_s;
    float r0_dx, fu, inv_r0;  // r0 / dx, D / r0, 1 / r0
    float eps, fk, tq, cs0;   // q dt / (2 m c), dt / (2 m c), q dt / (2 m), c dt / dx
    float sg;                 // charge sign of the current
    int pair;
    float cx, cy;             // scaled current per unit Esirkepov sum: x/z and y
    float* lam_pos;
    float* lam_u;
    float* lF;                // 6 float grids: the particles' scatter onto the field nodes
    const float* lj;          // 3 grids
    float* lam_nodes;
    double* grads;
    double inv_D;
};

__device__ __forceinline__ float hat_c(float d)
{
    const float a = fabsf(d);
    return a < 1.0f ? 1.0f - a : 0.0f;
}
__device__ __forceinline__ float dhat_c(float d) { return fabsf(d) < 1.0f ? (d > 0.0f ? -1.0f : 1.0f) : 0.0f; }

// staggered bilinear gather of a Yee component at (i + sx, k + sz) for a particle at cell (ci, ck),
// offsets (fx, fz); with lv != 0 also its transpose (node adjoints, position adjoints)
__device__ __forceinline__ float gather_stag(const FullAdjArgs& a, int f, int ci, int ck, float fx, float fz, float sx,
                                             float sz, float lv, float& lx, float& lz)
{
    const int nx = a.nx, nz = a.nz;
    float xs = fx - sx, fzz = fz - sz;
    int i = ci, k = ck;
    if (xs < 0.0f) { xs += 1.0f; i -= 1; }
    if (fzz < 0.0f) { fzz += 1.0f; k -= 1; }
    const int rows = sz > 0.0f ? nz : nz + 1;      // half-row components have nz rows
    bool clamped = false;
    if (k < 0) { k = 0; fzz = 0.0f; clamped = true; }
    else if (k > rows - 1 || (k == rows - 1 && fzz > 0.0f)) { k = rows - 1; fzz = 0.0f; clamped = true; }
    if (k >= rows - 1) { k = rows - 2; fzz = 1.0f; }
    const int i0 = i < 0 ? i + nx : i;
    const int i1 = i0 + 1 == nx ? 0 : i0 + 1;
    const float* A = a.F[f];
    const size_t r0 = (size_t)k * nx, r1 = r0 + nx;
    const float a00 = A[r0 + i0], a10 = A[r0 + i1], a01 = A[r1 + i0], a11 = A[r1 + i1];
    if (lv != 0.0f) {
        float* L = a.lF + (size_t)f * (nz + 1) * nx;
        atomicAdd(L + r0 + i0, lv * (1 - xs) * (1 - fzz));
        atomicAdd(L + r0 + i1, lv * xs * (1 - fzz));
        atomicAdd(L + r1 + i0, lv * (1 - xs) * fzz);
        atomicAdd(L + r1 + i1, lv * xs * fzz);
        lx += lv * ((1 - fzz) * (a10 - a00) + fzz * (a11 - a01));
        if (!clamped) lz += lv * ((1 - xs) * (a01 - a00) + xs * (a11 - a10));
    }
    return (1 - xs) * (1 - fzz) * a00 + xs * (1 - fzz) * a10 + (1 - xs) * fzz * a01 + xs * fzz * a11;
}

// transpose of the continuous Esirkepov current of one particle moving (x0, z0) -> (x1, z1) in
// coordinates local to its start cell (ci, ck): adds d/d(x0, z0, x1, z1, by) of sum lj * j into g
__device__ void cur_T(const FullAdjArgs& a, int ci, int ck, float x0, float z0, float x1, float z1, float by,
                      float g[5])
{
    const int nx = a.nx, nz = a.nz;
    const float bx = floorf(fminf(x0, x1)), bz = floorf(fminf(z0, z1));
    const int ib = ci + (int)bx, kb = ck + (int)bz;
    float S0x[3], S1x[3], S0z[3], S1z[3];
    float Lx[3][3], Ly[3][3], Lz[3][3];
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
            const size_t c = (size_t)(ok ? l : 0) * nx + ii;
            Lx[ia][b] = ok ? a.lj[c] : 0.0f;
            Ly[ia][b] = ok ? a.lj[nn + c] : 0.0f;
            Lz[ia][b] = ok ? a.lj[2 * nn + c] : 0.0f;
        }
    }
    const float cx = a.sg * a.cx, cy = a.sg * a.cy;
    float dS0x[3] = {0, 0, 0}, dS1x[3] = {0, 0, 0}, dS0z[3] = {0, 0, 0}, dS1z[3] = {0, 0, 0};
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const float Rx1 = Lx[1][b], Rx0 = Lx[0][b] + Lx[1][b], zsum = S0z[b] + S1z[b];
        dS1x[0] -= cx * zsum * Rx0; dS0x[0] += cx * zsum * Rx0;
        dS1x[1] -= cx * zsum * Rx1; dS0x[1] += cx * zsum * Rx1;
        const float zz = -cx * ((S1x[0] - S0x[0]) * Rx0 + (S1x[1] - S0x[1]) * Rx1);
        dS0z[b] += zz; dS1z[b] += zz;
    }
#pragma unroll
    for (int ia = 0; ia < 3; ia++) {
        const float Rz1 = Lz[ia][1], Rz0 = Lz[ia][0] + Lz[ia][1], xsum = S0x[ia] + S1x[ia];
        dS1z[0] -= cx * xsum * Rz0; dS0z[0] += cx * xsum * Rz0;
        dS1z[1] -= cx * xsum * Rz1; dS0z[1] += cx * xsum * Rz1;
        const float xx = -cx * ((S1z[0] - S0z[0]) * Rz0 + (S1z[1] - S0z[1]) * Rz1);
        dS0x[ia] += xx; dS1x[ia] += xx;
    }
    float gby = 0.0f;
#pragma unroll
    for (int ia = 0; ia < 3; ia++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const float L = Ly[ia][b] * cy;
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

// two fields with the same stagger pattern through one stencil (index, clamping, weights)
__device__ __forceinline__ void gather_stag2(const FullAdjArgs& a, int fA, int fB, int ci, int ck, float fx, float fz,
                                             float sx, float sz, float lvA, float lvB, float& lx, float& lz,
                                             float& vA, float& vB)
{
    const int nx = a.nx, nz = a.nz;
    float xs = fx - sx, fzz = fz - sz;
    int i = ci, k = ck;
    if (xs < 0.0f) { xs += 1.0f; i -= 1; }
    if (fzz < 0.0f) { fzz += 1.0f; k -= 1; }
    const int rows = sz > 0.0f ? nz : nz + 1;
    bool clamped = false;
    if (k < 0) { k = 0; fzz = 0.0f; clamped = true; }
    else if (k > rows - 1 || (k == rows - 1 && fzz > 0.0f)) { k = rows - 1; fzz = 0.0f; clamped = true; }
    if (k >= rows - 1) { k = rows - 2; fzz = 1.0f; }
    const int i0 = i < 0 ? i + nx : i;
    const int i1 = i0 + 1 == nx ? 0 : i0 + 1;
    const size_t r0 = (size_t)k * nx, r1 = r0 + nx;
    const float w00 = (1 - xs) * (1 - fzz), w10 = xs * (1 - fzz), w01 = (1 - xs) * fzz, w11 = xs * fzz;
    const size_t nn = (size_t)(nz + 1) * nx;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int f = h ? fB : fA;
        const float lv = h ? lvB : lvA;
        const float* A = a.F[f];
        const float a00 = A[r0 + i0], a10 = A[r0 + i1], a01 = A[r1 + i0], a11 = A[r1 + i1];
        if (lv != 0.0f) {
            float* L = a.lF + (size_t)f * nn;
            atomicAdd(L + r0 + i0, lv * w00);
            atomicAdd(L + r0 + i1, lv * w10);
            atomicAdd(L + r1 + i0, lv * w01);
            atomicAdd(L + r1 + i1, lv * w11);
            lx += lv * ((1 - fzz) * (a10 - a00) + fzz * (a11 - a01));
            if (!clamped) lz += lv * ((1 - xs) * (a01 - a00) + xs * (a11 - a10));
        }
        const float v = w00 * a00 + w10 * a10 + w01 * a01 + w11 * a11;
        if (h) vB = v; else vA = v;
    }
}


__global__ void __launch_bounds__(256, 2) k_adjoint_full(const FullAdjArgs a)
{
    __shared__ double sh[256];
    double gFF = 0.0, gR = 0.0;
    for (int64_t ch = blockIdx.x; ch * 256 < a.n; ch += gridDim.x) {
        const int64_t p = spread_index(ch);
        if (p >= a.n) continue;
        int ci, ck;
        split2(a.cell[p], a.nx, a.nx_magic, ci, ck);
        const float fx = a.fx[p], fz = a.fz[p];
        // ---- forward recompute (FP32, positions local to the cell) ----
        float E[3], B[3], dummy = 0.0f;
        gather_stag2(a, 0, 5, ci, ck, fx, fz, 0.5f, 0.0f, 0.0f, 0.0f, dummy, dummy, E[0], B[2]);
        gather_stag2(a, 2, 3, ci, ck, fx, fz, 0.0f, 0.5f, 0.0f, 0.0f, dummy, dummy, E[2], B[0]);
        E[1] = gather_stag(a, 1, ci, ck, fx, fz, 0.0f, 0.0f, 0.0f, dummy, dummy);
        B[1] = gather_stag(a, 4, ci, ck, fx, fz, 0.5f, 0.5f, 0.0f, dummy, dummy);
        DensAt d = {};
        PairD px = {0.0f, 0.0f, 0.0f, 0.0f}, pz = px;
        if (a.pair) {
            d = dens_at(a.rho, a.rho_s, a.nx, a.nz, ci, ck, fx, fz);
            px = pair_axis_d(d.n, d.qx, a.r0_dx, a.fu, a.inv_r0);
            pz = pair_axis_d(d.n, d.qz, a.r0_dx, a.fu, a.inv_r0);
        }
        const float Fp[3] = {px.F, 0.0f, pz.F};
        float um[3], t[3], sv[3], upr[3], uf[3];
        const float u0[3] = {a.ux[p], a.uy[p], a.uz[p]};
#pragma unroll
        for (int q = 0; q < 3; q++) um[q] = u0[q] + a.eps * E[q] + a.fk * Fp[q];
        const float gm = sqrtf(1.0f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        const float tfac = a.tq / gm;
#pragma unroll
        for (int q = 0; q < 3; q++) t[q] = tfac * B[q];
        const float t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
#pragma unroll
        for (int q = 0; q < 3; q++) sv[q] = 2.0f * t[q] / (1.0f + t2);
        upr[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
        upr[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
        upr[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
        uf[0] = um[0] + (upr[1] * sv[2] - upr[2] * sv[1]) + a.eps * E[0] + a.fk * Fp[0];
        uf[1] = um[1] + (upr[2] * sv[0] - upr[0] * sv[2]) + a.eps * E[1] + a.fk * Fp[1];
        uf[2] = um[2] + (upr[0] * sv[1] - upr[1] * sv[0]) + a.eps * E[2] + a.fk * Fp[2];
        const float g = sqrtf(1.0f + uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
        const float cs = a.cs0 / g;
        const float xl = fx + uf[0] * cs, zl = fz + uf[2] * cs;   // new position, local to (ci, ck)
        float z1 = zl, ufz_fin = uf[2];
        bool refl = false;
        if (ck == 0 && zl < 0.0f) { z1 = -zl; ufz_fin = -uf[2]; refl = true; }
        if (ck == a.nz - 1 && zl >= 1.0f) { z1 = 2.0f - zl; ufz_fin = -uf[2]; refl = true; }
        const float by = uf[1] / g;
        // ---- reverse ----
        float lx1 = a.lam_pos[2 * p], lz1 = a.lam_pos[2 * p + 1];
        float luf[3] = {a.lam_u[3 * p], a.lam_u[3 * p + 1], a.lam_u[3 * p + 2]};
        float lx0 = 0.0f, lz0 = 0.0f;
        if (a.sg != 0.0f) {
            float g5[5] = {0, 0, 0, 0, 0};
            cur_T(a, ci, ck, fx, fz, xl, z1, by, g5);
            lx0 += g5[0]; lz0 += g5[1]; lx1 += g5[2]; lz1 += g5[3];
            const float ig = 1.0f / g, ig3 = ig * ig * ig;
            luf[0] -= g5[4] * uf[1] * uf[0] * ig3;
            luf[1] += g5[4] * (ig - uf[1] * uf[1] * ig3);
            luf[2] -= g5[4] * uf[1] * ufz_fin * ig3;
        }
        float lzn = lz1;
        if (refl) { lzn = -lz1; luf[2] = -luf[2]; }
        const float udl = (uf[0] * lx1 + uf[2] * lzn) / (g * g);
        float lu[3];
        lu[0] = luf[0] + cs * (lx1 - uf[0] * udl);
        lu[1] = luf[1] + cs * (0.0f - uf[1] * udl);
        lu[2] = luf[2] + cs * (lzn - uf[2] * udl);
        lx0 += lx1;
        lz0 += lzn;
        // Boris transpose
        float la[3], lum[3], lupr[3], lsv[3], lt[3];
#pragma unroll
        for (int q = 0; q < 3; q++) { la[q] = lu[q]; lum[q] = lu[q]; }
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
        const float tl = t[0] * lsv[0] + t[1] * lsv[1] + t[2] * lsv[2], d1 = 1.0f / (1.0f + t2);
#pragma unroll
        for (int q = 0; q < 3; q++) lt[q] += 2.0f * lsv[q] * d1 - 4.0f * tl * t[q] * d1 * d1;
        float lB[3], ltf = 0.0f;
#pragma unroll
        for (int q = 0; q < 3; q++) { lB[q] = tfac * lt[q]; ltf += B[q] * lt[q]; }
        const float lgm = -tfac / gm * ltf;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            lum[q] += lgm * um[q] / gm;
            la[q] += lum[q];
        }
        a.lam_u[3 * p] = lum[0];
        a.lam_u[3 * p + 1] = lum[1];
        a.lam_u[3 * p + 2] = lum[2];
        // field gathers
        {
            float t0, t1;
            gather_stag2(a, 0, 5, ci, ck, fx, fz, 0.5f, 0.0f, a.eps * la[0], lB[2], lx0, lz0, t0, t1);
            gather_stag2(a, 2, 3, ci, ck, fx, fz, 0.0f, 0.5f, a.eps * la[2], lB[0], lx0, lz0, t0, t1);
            gather_stag(a, 1, ci, ck, fx, fz, 0.0f, 0.0f, a.eps * la[1], lx0, lz0);
            gather_stag(a, 4, ci, ck, fx, fz, 0.5f, 0.5f, lB[1], lx0, lz0);
        }
        if (a.pair) pair_T(d, px, pz, a.fk * la[0], a.fk * la[2], a.inv_r0, a.nx, a.lam_nodes, lx0, lz0, gFF, gR);
        a.lam_pos[2 * p] = lx0;
        a.lam_pos[2 * p + 1] = lz0;
    }
    if (a.pair) {
        const double sD = block_sum_d(gFF, sh), sR = block_sum_d(gR, sh);
        if (threadIdx.x == 0) {
            atomicAdd(a.grads, sD * a.inv_D);
            atomicAdd(a.grads + 1, sR);
        }
    }
}

__global__ void k_adjoint_seed_u(int64_t n, const float* ux, const float* uy, const float* uz, float kin_mc2w,
                                 float* lam_pos, float* lam_u)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const float x = ux[p], y = uy[p], z = uz[p];
        const float ig = kin_mc2w / sqrtf(1.0f + x * x + y * y + z * z);
        lam_u[3 * p] = ig * x;
        lam_u[3 * p + 1] = ig * y;
        lam_u[3 * p + 2] = ig * z;
        lam_pos[2 * p] = 0.0f;
        lam_pos[2 * p + 1] = 0.0f;
    }
}

// the particles' FP32 scatter added into the FP64 field adjoints
__global__ void k_fold_scatter(double* __restrict__ lF, const float* __restrict__ scatter, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        lF[q] += (double)scatter[q];
}

static FullAdjArgs make_full_adj(Ctx& c, int s, float* const* lam_pos, float* const* lam_u, float* lam_nodes,
                                 float* lF, const float* lj, double* grads)
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
    a.rho_s = (float)c.rho_scale;
    a.r0_dx = (float)(c.r0 / c.cfg.dx);
    a.fu = (float)(c.D / c.r0);
    a.inv_r0 = (float)(1.0 / c.r0);
    const double q = s == 0 ? c.cfg.ion_charge * kQe : -kQe;
    a.eps = (float)(q * c.dt / (2.0 * S.mass * kC));
    a.fk = (float)(c.dt / (2.0 * S.mass * kC));
    a.tq = (float)(q * c.dt / (2.0 * S.mass));
    a.cs0 = (float)(kC * c.dt / c.cfg.dx);
    a.sg = (float)S.jsign;
    a.pair = S.pair;
    a.cx = (float)(kQe * c.w / (2.0 * c.cfg.dx * kEps0));
    a.cy = (float)(kQe * c.w * kC * c.dt / (6.0 * c.cfg.dx * c.cfg.dx * kEps0));
    a.lam_pos = lam_pos[s];
    a.lam_u = lam_u[s];
    a.lF = lF;
    a.lj = lj;
    a.lam_nodes = lam_nodes;
    a.grads = grads;
    a.inv_D = 1.0 / c.D;
    return a;
}

void launch_adjoint_seed_full(Ctx& c, double kin, const double* w_nodes, float* const* lam_pos, float* const* lam_u,
                              float* lam_nodes, double* lF, float* lj, double* r0_out, cudaStream_t st)
{
    const size_t nn = c.nn;
    cudaMemsetAsync(lF, 0, sizeof(double) * 9 * nn, st);
    cudaMemsetAsync(lj, 0, sizeof(float) * 3 * nn, st);
    for (int s = 0; s < c.nsp; s++) {
        const Species& S = c.sp[s];
        if (s == 0 && S.pair) continue;          // seeded with its density below
        k_adjoint_seed_u<<<agrid(c, S.n), 256, 0, st>>>(S.n, S.a.ux, S.a.uy, S.a.uz,
                                                         (float)(kin * c.w * S.mass * kC * kC), lam_pos[s], lam_u[s]);
    }
    if (c.sp[0].pair) seed_pair_species(c, kin, w_nodes, lam_pos[0], lam_u[0], lam_nodes, r0_out, st);
}

void launch_adjoint_step_full(Ctx& c, float* const* lam_pos, float* const* lam_u, float* lam_nodes, double* lF,
                              float* lj, double* grads, cudaStream_t st)
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
    if (c.sp[0].pair) cudaMemsetAsync(lam_nodes, 0, sizeof(float) * nn, st);
    float* scatter = reinterpret_cast<float*>(lF + 6 * nn);        // six float grids
    cudaMemsetAsync(scatter, 0, sizeof(float) * 6 * nn, st);
    for (int s = 0; s < c.nsp; s++) {
        FullAdjArgs a = make_full_adj(c, s, lam_pos, lam_u, lam_nodes, scatter, lj, grads);
        if (a.n > 0) k_adjoint_full<<<agrid(c, a.n), 256, 0, st>>>(a);
    }
    k_fold_scatter<<<agrid(c, (int64_t)(6 * nn)), 256, 0, st>>>(lF, scatter, (int64_t)(6 * nn));
    if (c.sp[0].pair) {
        AdjArgs b = make_adj(c, 0, lam_pos[0], lam_u[0], lam_nodes, grads);
        k_adjoint_b<<<agrid(c, b.n), 256, 0, st>>>(b);
    }
}

}  // namespace gbpic
