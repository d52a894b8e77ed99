// Device-side building blocks of the PIC cycle: interpolation back to the particle, the
// pair-potential force of Eqs. (1)-(3), the Boris push and fixed-point shapes.
#pragma once

#include "pic_internal.cuh"

namespace gbpic {

__device__ __forceinline__ int wrap_x(int i, int nx) { return i < 0 ? i + nx : (i >= nx ? i - nx : i); }

// Pair-species node sum with the wall rows doubled (mirror image of the slab behind a wall).
__device__ __forceinline__ long long rho_node(const u64* __restrict__ rho, int nx, int nz, int i, int k)
{
    long long v = (long long)__ldg(rho + (size_t)k * nx + i);
    return (k == 0 || k == nz) ? 2 * v : v;
}

// Node density (units n0) and its gradient (units n0 per cell) at a particle in cell (i, k) with
// offsets (fx, fz): bilinear density; the gradient is the edge difference of the node density
// interpolated along the other axis, i.e. the exact gradient of the bilinear density.
// Differences are taken in integers before the single rounding to FP32.
__device__ __forceinline__ void gather_density(const u64* __restrict__ rho, int nx, int nz, float rho_s,
                                               int i, int k, float fx, float fz,
                                               float& n, float& dnx, float& dnz)
{
    int i1 = wrap_x(i + 1, nx);
    long long r00 = rho_node(rho, nx, nz, i, k), r10 = rho_node(rho, nx, nz, i1, k);
    long long r01 = rho_node(rho, nx, nz, i, k + 1), r11 = rho_node(rho, nx, nz, i1, k + 1);
    float gx = 1.0f - fx, gz = 1.0f - fz;
    float a00 = (float)r00, a10 = (float)r10, a01 = (float)r01, a11 = (float)r11;
    n = rho_s * (gz * (gx * a00 + fx * a10) + fz * (gx * a01 + fx * a11));
    dnx = rho_s * (gz * (float)(r10 - r00) + fz * (float)(r11 - r01));
    dnz = rho_s * (gx * (float)(r01 - r00) + fx * (float)(r11 - r10));
}

// Lennard-Jones derivative U'(r) (units D/r0) from inv = r0 / r.
__device__ __forceinline__ float lj_dU_inv(float inv)
{
    float i2 = inv * inv, i6 = i2 * i2 * i2;
    return 12.0f * i6 * inv * (1.0f - i6);
}
__device__ __forceinline__ float lj_U_inv(float inv)
{
    float i2 = inv * inv, i6 = i2 * i2 * i2;
    return i6 * (i6 - 2.0f);
}

// Branch factor of the altered potential: s_rep inside r0 (inv > 1), c_att outside.
__device__ __forceinline__ float branch(int pot_mode, float c_att, float s_rep, float inv)
{
    return (pot_mode & 3) == 0 ? 1.0f : (inv > 1.0f ? s_rep : c_att);
}

// approximate transcendental helpers (hardware ex2 / lg2 / rcp, relative error ~1e-7)
__device__ __forceinline__ float fast_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float fast_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// n^(1/3) for n > 0
__device__ __forceinline__ float fast_cbrt(float n) { return fast_ex2(fast_lg2(n) * (1.0f / 3.0f)); }

// e^x from the hardware base-2 exponential, ex2(x log2 e): relative error ~2^-22 plus the rounding
// of x log2 e (~|x| 2^-24), below 3e-6 for the |x| < 40 the pair potentials take
__device__ __forceinline__ float exp_hw(float x) { return fast_ex2(x * 1.44269504088896341f); }
// ln x from the hardware base-2 logarithm (absolute error ~1e-7 for x near 1)
__device__ __forceinline__ float log_hw(float x) { return fast_lg2(x) * 0.693147180559945309f; }
// e^x - 1 without cancellation: for |x| < 1/2 its Taylor series to x^9 / 9! (the first omitted
// term is below 3e-10 of the sum), else exp_hw(x) - 1 (at most e^(1/2) / (e^(1/2) - 1) ~ 2.5 times
// the relative error of exp_hw)
__device__ __forceinline__ float expm1_hw(float x)
{
    if (fabsf(x) < 0.5f) {
        float p = 2.75573192e-6f;                // 1 / 9!
        p = fmaf(p, x, 2.48015873e-5f);          // 1 / 8!
        p = fmaf(p, x, 1.98412698e-4f);          // 1 / 7!
        p = fmaf(p, x, 1.38888889e-3f);          // 1 / 6!
        p = fmaf(p, x, 8.33333333e-3f);          // 1 / 5!
        p = fmaf(p, x, 4.16666667e-2f);          // 1 / 4!
        p = fmaf(p, x, 1.66666667e-1f);          // 1 / 3!
        p = fmaf(p, x, 0.5f);
        p = fmaf(p, x, 1.0f);
        return x * p;
    }
    return exp_hw(x) - 1.0f;
}

// Morse potential (pot_mode 2; the paper's mapping of density to neighbour distance takes any pair
// potential): U = E^2 - 2E, E = exp(-a (r - 1)), units D with r in r0; minimum -1 at r = 1 like
// Eq. (3). The pair functions below take the stiffness a in their c_att argument.
__device__ __forceinline__ float morse_U_inv(float inv, float a)
{
    const float e = exp_hw(-a * (1.0f / inv - 1.0f));
    return e * (e - 2.0f);
}
__device__ __forceinline__ float morse_dU_inv(float inv, float a)    // U'(r), units D / r0
{
    const float e = exp_hw(-a * (1.0f / inv - 1.0f));
    return 2.0f * a * e * (1.0f - e);
}

// Eq. (3)'s force difference for the Morse form: with both neighbours finite
//   U'(r+) - U'(r-) = 2a (E+ - E-) (1 - E+ - E-),  E+ - E- = E- expm1(-a (r+ - r-)),
//   r+ - r- = 2h / (c (1 - h^2)),
// free of cancellation. Inlined into the kernel instances that compile the Morse form in (an
// out-of-line call cost the transport kernel its registers' round trips through local memory:
// 0.165 -> 0.196 ms per launch on the crater slab once the call site changed); the run-time
// dispatch of the diagnostics calls the out-of-line copy below.
__device__ __forceinline__ float morse_axis_inl(float c, float h, float a)
{
    const float ip = c * (1.0f - h), im = c * (1.0f + h);
    if (ip > 0.0f && im > 0.0f) {
        const float ep = exp_hw(-a * (1.0f / ip - 1.0f)), em = exp_hw(-a * (1.0f / im - 1.0f));
        const float dr = 2.0f * h / (c * (1.0f - h * h));
        return 2.0f * a * em * expm1_hw(-a * dr) * (1.0f - ep - em);
    }
    float f = 0.0f;
    if (ip > 0.0f) f += morse_dU_inv(ip, a);
    if (im > 0.0f) f -= morse_dU_inv(im, a);
    return f;
}

static __device__ __noinline__ float morse_axis(float c, float h, float a) { return morse_axis_inl(c, h, a); }

// Pair energy U(r) (units D) of one neighbour at r0 / r = inv under pot_mode.
__device__ __forceinline__ float pair_U(int pot_mode, float c_att, float s_rep, float inv)
{
    return (pot_mode & 3) == 2 ? morse_U_inv(inv, c_att) : branch(pot_mode, c_att, s_rep, inv) * lj_U_inv(inv);
}

// Dimensionless pair force along one axis (units D / r0) on an atom at local density n (> 0)
// with c = n^(1/3) and gradient dn along that axis.
//   Eq. (1): g = d rbar / dx = -(1/3) (r0 / dx) n^(-4/3) dn;  h = g / 2
//   Eq. (2): neighbour distances rbar / (1 -+ h) -> r0 / dist = c (1 -+ h)
//   Eq. (3): F = U'(dist+) - U'(dist-).
// With both neighbours finite and on the same branch the difference is evaluated without
// cancellation: (1-h)^p - (1+h)^p = -2 P_p(h), P_p the odd part of (1+h)^p, so
//   F = 24 [ c n^4 P13(h) - c n^2 P7(h) ].
// ZERO_SKIP: a branch whose factor is 0 contributes nothing even where U' overflows FP32 (a
// neighbour pulled arbitrarily close at the vacuum edge); the probe calls of the calibration use it.
// POT: the potential code compiled in (bits 0-1 the potential, bit 2 the HCP lattice). kPotLJ: Eq. (3)
// as printed (pot_mode 0); kPotAlt: the altered potential (pot_mode 1); kPotMorse: the Morse form
// (pot_mode 2); kPotRuntime: the code is read from pot_mode at run time (diagnostics). The particle
// kernels take the code as a template argument, so that the plain Lennard-Jones instances carry no
// branch factor, Morse or HCP code (a uniform run-time branch to the out-of-line Morse call cost 6 %
// of the 3D particle kernel's time).
enum { kPotRuntime = -1, kPotLJ = 0, kPotAlt = 1, kPotMorse = 2, kPotEam = 3, kLatHcp = 4 };

// kPotEam: the embedded-atom form (pot_mode 3, cubic lattice only; see eam_forces below).
// The kernel instance code of a run-time potential code (pot_mode in bits 0-1, kLatHcp in bit 2).
inline int pot_instance(int code) { return code & 7; }

template <bool ZERO_SKIP = false, int POT = kPotRuntime>
__device__ __forceinline__ float pair_axis(float n, float c, float inv43, float dn, float h_coef,
                                           int pot_mode, float c_att, float s_rep)
{
    float h = -h_coef * dn * inv43;
    if (POT >= 0 && (POT & 3) == kPotMorse) return morse_axis_inl(c, h, c_att);
    if (POT == kPotRuntime && (pot_mode & 3) == 2) return morse_axis(c, h, c_att);
    const int pm = POT >= 0 ? (POT & 3) : pot_mode;
    float ip = c * (1.0f - h);      // r0 / dist to the neighbour on the + side
    float im = c * (1.0f + h);      // r0 / dist to the neighbour on the - side
    if (ip > 0.0f && im > 0.0f) {
        float fp = branch(pm, c_att, s_rep, ip), fm = branch(pm, c_att, s_rep, im);
        if (ZERO_SKIP && fp != fm)
            return (fp != 0.0f ? fp * lj_dU_inv(ip) : 0.0f) - (fm != 0.0f ? fm * lj_dU_inv(im) : 0.0f);
        float h2 = h * h;
        float p7 = h * (7.0f + h2 * (35.0f + h2 * (21.0f + h2)));
        float p13 = h * (13.0f + h2 * (286.0f + h2 * (1287.0f + h2 * (1716.0f + h2 * (715.0f + h2 * (78.0f + h2))))));
        float n2 = n * n;
        const float d = 24.0f * c * n2 * (n2 * p13 - p7);     // U'(dist+) - U'(dist-), no cancellation
        if (fp == fm) return fp * d;
        // the neighbours on different branches of the altered potential:
        // fp U'(+) - fm U'(-) = fp (U'(+) - U'(-)) + (fp - fm) U'(-), neither term cancelling
        return fp * d + (fp - fm) * lj_dU_inv(im);
    }
    float f = 0.0f;
    if (ip > 0.0f) {
        const float fp = branch(pm, c_att, s_rep, ip);
        if (!ZERO_SKIP || fp != 0.0f) f += fp * lj_dU_inv(ip);
    }
    if (im > 0.0f) {
        const float fm = branch(pm, c_att, s_rep, im);
        if (!ZERO_SKIP || fm != 0.0f) f -= fm * lj_dU_inv(im);
    }
    return f;
}

// Pair energy per atom (units D): half the sum of U over the six neighbours.
__device__ __forceinline__ float pair_energy_axis(float c, float inv43, float dn, float h_coef,
                                                  int pot_mode, float c_att, float s_rep)
{
    float h = -h_coef * dn * inv43;
    float ip = c * (1.0f - h), im = c * (1.0f + h);
    float e = 0.0f;
    if (ip > 0.0f) e += pair_U(pot_mode, c_att, s_rep, ip);
    if (im > 0.0f) e += pair_U(pot_mode, c_att, s_rep, im);
    return e;
}

// Staggered bilinear field gather. (hx, hz) = 1 when the component sits half a cell up in x / z.
// Half-row components exist on rows 0..nz-1; positions outside that range take the edge row.
__device__ __forceinline__ float gather_field(const float* __restrict__ A, int nx, int nz, int i, int k,
                                              float fx, float fz, int hx, int hz)
{
    int i0 = i;
    float wx = fx;
    if (hx) {
        if (fx >= 0.5f) { wx = fx - 0.5f; }
        else { i0 = wrap_x(i - 1, nx); wx = fx + 0.5f; }
    }
    int i1 = wrap_x(i0 + 1, nx);
    int r0 = k, r1 = k + 1;
    float wz = fz;
    if (hz) {
        if (fz >= 0.5f) {
            wz = fz - 0.5f;
            if (k >= nz - 1) { r0 = nz - 2; r1 = nz - 1; wz = 1.0f; }
        } else if (k >= 1) {
            r0 = k - 1; r1 = k; wz = fz + 0.5f;
        } else {
            r0 = 0; r1 = 1; wz = 0.0f;
        }
    }
    const float* row0 = A + (size_t)r0 * nx;
    const float* row1 = A + (size_t)r1 * nx;
    float a = __ldg(row0 + i0), b = __ldg(row0 + i1), cc = __ldg(row1 + i0), d = __ldg(row1 + i1);
    return (1.0f - wz) * ((1.0f - wx) * a + wx * b) + wz * ((1.0f - wx) * cc + wx * d);
}

// Relativistic Boris push of u = gamma v / c with the pair force added to both half kicks.
__device__ __forceinline__ void boris(float& ux, float& uy, float& uz, float ex, float ey, float ez,
                                      float bx, float by, float bz, float e_kick, float b_rot)
{
    ux += e_kick * ex; uy += e_kick * ey; uz += e_kick * ez;
    float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
    float tx = b_rot * ig * bx, ty = b_rot * ig * by, tz = b_rot * ig * bz;
    float s = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
    float px = ux + (uy * tz - uz * ty);
    float py = uy + (uz * tx - ux * tz);
    float pz = uz + (ux * ty - uy * tx);
    ux += s * (py * tz - pz * ty);
    uy += s * (pz * tx - px * tz);
    uz += s * (px * ty - py * tx);
    ux += e_kick * ex; uy += e_kick * ey; uz += e_kick * ez;
}

// J_y code V = rint(beta_y 2^b), beta_y = u_y / gamma, taken in FP32 with explicit rounding (no
// fused multiply-add) so that it is reproducible outside the GPU; scale = 2^b (b = 18 unless the
// slab's particles per cell call for a coarser code, see choose_jy_bits). For u^2 < 2^-10 the
// inverse Lorentz factor is the series 1 - u^2 (1/2 - 3/8 u^2) (next term 5/16 u^6 < 3e-10);
// otherwise it is 1 / sqrt(1 + u^2) with IEEE square root and division.
__device__ __forceinline__ int jy_code(float ux, float uy, float uz, float scale)
{
    float u2 = __fmul_rn(ux, ux);
    u2 = __fadd_rn(u2, __fmul_rn(uy, uy));
    u2 = __fadd_rn(u2, __fmul_rn(uz, uz));
    float by;
    if (u2 < 0.0009765625f) {
        float t = __fmul_rn(u2, 0.375f);
        t = __fsub_rn(0.5f, t);
        t = __fmul_rn(u2, t);
        by = __fmul_rn(uy, __fsub_rn(1.0f, t));
    } else {
        by = __fdiv_rn(uy, __fsqrt_rn(__fadd_rn(1.0f, u2)));
    }
    return __float2int_rn(__fmul_rn(by, scale));
}

// Fixed-point offset Q(f) = rint(f 2^16) in [0, 2^16].
__device__ __forceinline__ int qoff(float f) { return __float2int_rn(f * 65536.0f); }

// Linear (hat) weights of a fixed-point coordinate d (relative to node 0 of a 3-node stencil,
// 0 <= d <= 2^17) on nodes 0, 1, 2.
__device__ __forceinline__ void hat3(int d, int& s0, int& s1, int& s2)
{
    s0 = max(0, kQOne - d);
    s1 = kQOne - abs(d - kQOne);
    s2 = max(0, d - kQOne);
}

}  // namespace gbpic

namespace gbpic {

// Pair-potential half kick components (units D / r0) along x and z at local density n (units
// n0) with gradient (dnx, dnz) per cell: Eqs. (1)-(3) via pair_axis.
// HCP (ideal axial ratio, c axis along z, sublattices averaged) in the x-z plane of a y-uniform state:
// the twelve neighbours pair up with their opposites into directions (1, 0) (weight 1), (1/2, 0)
// (the two basal pairs at +-60 degrees, weight 2) and (e, s) with e = 1/2, 0, -1/2, s = sqrt(2/3)
// (weight 1 each); a pair along the unit vector u contributes (U'(r+) - U'(r-)) u, r+- from Eq. (2)
// with the density derivative along u. Their y components cancel.
constexpr float kHcpS = 0.816496580927726f;    // sqrt(2/3)

// ---- the embedded-atom form (pot_mode 3) on the cubic lattice (the paper: other potentials are
// readily adapted to its mapping of density to neighbour distance). Atom i's embedding density is
// the sum of f over its six Eq. (2) neighbours; neighbour j's own is 6 f(n_j^(-1/3)), n_j the
// interpolated density at j's position taken along the axis, n + s dn (s = the neighbour's offset
// in cells: its distance in r0 times r0 / dx = 6 h_coef), but never less than f(r), the density of
// its bond back to the atom; each bond pulls with T = phi'(r) + (F'(rho_i) + F'(rho_j)) f'(r) and
// the force along an axis is T(r+) - T(r-).
__device__ __forceinline__ float eam_f(const EamP& e, float r) { return exp_hw(-e.beta * (r - 1.0f)); }
__device__ __forceinline__ float eam_phi(const EamP& e, float r) { return e.phi * exp_hw(-e.gamma * (r - 1.0f)); }
// dF / d rho
__device__ __forceinline__ float eam_dF(const EamP& e, float rho)
{
    if (!(rho > 0.0f)) return 0.0f;
    const float lx = log_hw(rho * (1.0f / 6.0f)), k = e.alpha / e.beta, m = e.gamma / e.beta;
    return (e.ec * k * k * lx * exp_hw((k - 1.0f) * lx) - 3.0f * e.phi * m * exp_hw((m - 1.0f) * lx)) * (1.0f / 6.0f);
}
__device__ __forceinline__ float eam_F(const EamP& e, float rho)
{
    if (!(rho > 0.0f)) return 0.0f;
    const float lx = log_hw(rho * (1.0f / 6.0f)), k = e.alpha / e.beta, m = e.gamma / e.beta;
    return -e.ec * (1.0f - k * lx) * exp_hw(k * lx) - 3.0f * e.phi * exp_hw(m * lx);
}

// F'(rho) of a neighbour whose own environment is uniform at spacing rb (rho = 6 f(rb)), as a
// function of rb: with L = ln(rho / 6) = -beta (rb - 1),
//   F' = -(1/6) [ec k^2 beta (rb - 1) e^(-(alpha - beta)(rb - 1)) + 3 phi m e^(-(gamma - beta)(rb - 1))].
__device__ __forceinline__ float eam_dF_rb(const EamP& e, float rb)
{
    const float k = e.alpha / e.beta, m = e.gamma / e.beta, t = rb - 1.0f;
    return -(1.0f / 6.0f) *
           (e.ec * k * k * e.beta * t * exp_hw(-(e.alpha - e.beta) * t) + 3.0f * e.phi * m * exp_hw(-(e.gamma - e.beta) * t));
}

// F'(rb+) - F'(rb-) from rb- and dl = rb+ - rb- without cancellation (expm1 of the exponents'
// differences; the (rb - 1) factor moves by dl).
__device__ __forceinline__ float eam_dF_rb_diff(const EamP& e, float rbm, float dl)
{
    const float k = e.alpha / e.beta, m = e.gamma / e.beta, t = rbm - 1.0f;
    const float a = e.alpha - e.beta, b = e.gamma - e.beta;
    const float ea = exp_hw(-a * t), eb = exp_hw(-b * t);
    const float d1 = t * expm1_hw(-a * dl) + dl * exp_hw(-a * dl);        // (t + dl) e^(-a dl) - t
    return -(1.0f / 6.0f) * (e.ec * k * k * e.beta * ea * d1 + 3.0f * e.phi * m * eb * expm1_hw(-b * dl));
}

// Force (units D / r0) along the axes and energy (units D, the atom's full share: the callers
// that halve pair energies get twice it) of an atom at density n (c = n^(1/3), inv43 = n^(-4/3))
// with gradient g per cell. NAX axes carry Eq. (2) neighbours (2: x and z, g[1] unused, the +-y
// neighbours at rbar with their own density n; 3: x, y, z). With both neighbours of an axis
// finite, inside the slab and with their own densities above their bonds' (the floor inactive),
// T(r+) - T(r-) is formed without cancellation:
//   -gamma [phi(r+) - phi(r-)] - beta F'_i [f(r+) - f(r-)] - beta [(F'_+ - F'_-) f(r+) + F'_- (f(r+) - f(r-))],
//   phi(r+) - phi(r-) = phi(r-) expm1(-gamma dr), f(r+) - f(r-) = f(r-) expm1(-beta dr),
//   dr = r+ - r- = 2h / (c (1 - h^2)), and F'_+ - F'_- from the neighbours' spacings, whose
//   difference is (n-^(1/3) - n+^(1/3)) / (n+ n-)^(1/3) with n+^(1/3) - n-^(1/3) = (n+ - n-) / (sum
//   of the three products of their cube roots), n+ - n- = s (r+ + r-) dn.
template <int NAX>
__device__ __forceinline__ void eam_forces(const EamP& e, float n, float c, float inv43, const float g[3], float h_coef,
                                           float F[3], float* u)
{
    constexpr int nax = 3;
    float rp[nax], rm[nax], hh[nax], rho = 0.0f, up = 0.0f;
#pragma unroll
    for (int d = 0; d < nax; d++) {
        hh[d] = 0.0f;
        if (NAX == 2 && d == 1) {
            rp[d] = rm[d] = 1.0f / c;
        } else {
            const float h = -h_coef * g[d] * inv43;
            const float ip = c * (1.0f - h), im = c * (1.0f + h);
            hh[d] = h;
            rp[d] = ip > 0.0f ? 1.0f / ip : 0.0f;        // 0: the neighbour is at infinity
            rm[d] = im > 0.0f ? 1.0f / im : 0.0f;
        }
        if (rp[d] > 0.0f) { rho += eam_f(e, rp[d]); up += eam_phi(e, rp[d]); }
        if (rm[d] > 0.0f) { rho += eam_f(e, rm[d]); up += eam_phi(e, rm[d]); }
    }
    const float dFi = eam_dF(e, rho), s = 6.0f * h_coef, ln6b = 1.791759469f / e.beta;
#pragma unroll
    for (int d = 0; d < nax; d++) {
        F[d] = 0.0f;
        if (NAX == 2 && d == 1) continue;
        const float npl = n + rp[d] * s * g[d], nmi = n - rm[d] * s * g[d];
        if (rp[d] > 0.0f && rm[d] > 0.0f && npl > 0.0f && nmi > 0.0f) {
            const float cp = fast_cbrt(npl), cm = fast_cbrt(nmi);
            // both neighbours' own densities 6 f(rb) above their bonds' f(r) (rb <= r + ln 6 / beta):
            // the floor below is inactive
            if (cp * (rp[d] + ln6b) >= 1.0f && cm * (rm[d] + ln6b) >= 1.0f) {
                const float h = hh[d];
                const float dr = 2.0f * h / (c * (1.0f - h * h));
                const float rbm = 1.0f / cm;
                // rb+ - rb- = (cm - cp) / (cp cm), cp - cm = (n+ - n-) / (cp^2 + cp cm + cm^2)
                const float dn = (rp[d] + rm[d]) * s * g[d];
                const float dl = -dn / ((cp * cp + cp * cm + cm * cm) * cp * cm);
                const float fm = eam_f(e, rm[d]), fp = eam_f(e, rp[d]), df = fm * expm1_hw(-e.beta * dr);
                const float dFm = eam_dF_rb(e, rbm);
                F[d] = -e.gamma * eam_phi(e, rm[d]) * expm1_hw(-e.gamma * dr) - e.beta * dFi * df -
                       e.beta * (eam_dF_rb_diff(e, rbm, dl) * fp + dFm * df);
                continue;
            }
        }
        float T[2] = {0.0f, 0.0f};
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const float r = side == 0 ? rp[d] : rm[d];
            if (!(r > 0.0f)) continue;
            const float nj = side == 0 ? npl : nmi, fr = eam_f(e, r);
            // the neighbour holds at least its bond back to the atom: rho_j >= f(r) (a neighbour
            // density from n_j alone diverges F' as n_j -> 0 at a free surface)
            const float rhoj = fmaxf(nj > 0.0f ? 6.0f * eam_f(e, 1.0f / fast_cbrt(nj)) : 0.0f, fr);
            T[side] = -e.gamma * eam_phi(e, r) - e.beta * (dFi + eam_dF(e, rhoj)) * fr;
        }
        F[d] = T[0] - T[1];
    }
    if (u) *u = eam_F(e, rho) + 0.5f * up;
}

template <bool ZERO_SKIP = false, int POT = kPotRuntime>
__device__ __forceinline__ void pair_force_xz(float n, float dnx, float dnz, float h_coef, int pot_mode, float c_att,
                                              float s_rep, float& fx, float& fz, const EamP& eam = EamP{})
{
    fx = 0.0f;
    fz = 0.0f;
    if (n > 0.0f) {
        const float c = fast_cbrt(n);
        const float inv43 = fast_rcp(n * c);
        if ((POT >= 0 && (POT & 3) == kPotEam) || (POT == kPotRuntime && (pot_mode & 3) == 3)) {
            const float g[3] = {dnx, 0.0f, dnz};
            float F[3];
            eam_forces<2>(eam, n, c, inv43, g, h_coef, F, nullptr);
            fx = F[0];
            fz = F[2];
            return;
        }
        const bool hcp = POT >= 0 ? (POT & kLatHcp) != 0 : (pot_mode & kLatHcp) != 0;
        if (!hcp) {
            fx = pair_axis<ZERO_SKIP, POT>(n, c, inv43, dnx, h_coef, pot_mode, c_att, s_rep);
            fz = pair_axis<ZERO_SKIP, POT>(n, c, inv43, dnz, h_coef, pot_mode, c_att, s_rep);
        } else {
            const float a1 = pair_axis<ZERO_SKIP, POT>(n, c, inv43, dnx, h_coef, pot_mode, c_att, s_rep);
            const float a2 = pair_axis<ZERO_SKIP, POT>(n, c, inv43, 0.5f * dnx, h_coef, pot_mode, c_att, s_rep);
            const float bp = pair_axis<ZERO_SKIP, POT>(n, c, inv43, 0.5f * dnx + kHcpS * dnz, h_coef, pot_mode, c_att,
                                                       s_rep);
            const float b0 = pair_axis<ZERO_SKIP, POT>(n, c, inv43, kHcpS * dnz, h_coef, pot_mode, c_att, s_rep);
            const float bm = pair_axis<ZERO_SKIP, POT>(n, c, inv43, -0.5f * dnx + kHcpS * dnz, h_coef, pot_mode, c_att,
                                                       s_rep);
            fx = a1 + a2 + 0.5f * (bp - bm);
            fz = kHcpS * (bp + b0 + bm);
        }
    }
}

// Eq. (3) as printed on the cubic lattice, both in-plane axes at once: the cancellation-free form of
// pair_axis evaluated on (x, z) pairs with packed FP32x2 arithmetic (one instruction per pair).
// Falls back to pair_axis when a neighbour sits at infinity on either axis (|h| >= 1).
__device__ __forceinline__ void lj_pair_xz2(float n, float dnx, float dnz, float h_coef, float& fx, float& fz)
{
    fx = 0.0f;
    fz = 0.0f;
    if (!(n > 0.0f)) return;
    const float c = fast_cbrt(n);
    const float inv43 = fast_rcp(n * c);
    const float hx = -h_coef * dnx * inv43, hz = -h_coef * dnz * inv43;
    if (fabsf(hx) < 1.0f && fabsf(hz) < 1.0f) {
        const float2 h = make_float2(hx, hz);
        const float2 h2 = __fmul2_rn(h, h);
        float2 t = __fadd2_rn(h2, make_float2(21.0f, 21.0f));
        t = __ffma2_rn(h2, t, make_float2(35.0f, 35.0f));
        t = __ffma2_rn(h2, t, make_float2(7.0f, 7.0f));
        const float2 p7 = __fmul2_rn(h, t);
        float2 u = __fadd2_rn(h2, make_float2(78.0f, 78.0f));
        u = __ffma2_rn(h2, u, make_float2(715.0f, 715.0f));
        u = __ffma2_rn(h2, u, make_float2(1716.0f, 1716.0f));
        u = __ffma2_rn(h2, u, make_float2(1287.0f, 1287.0f));
        u = __ffma2_rn(h2, u, make_float2(286.0f, 286.0f));
        u = __ffma2_rn(h2, u, make_float2(13.0f, 13.0f));
        const float2 p13 = __fmul2_rn(h, u);
        // 24 c n^2 (n^2 P13 - P7)
        const float n2 = n * n, s = 24.0f * c * n2;
        const float2 d = __ffma2_rn(make_float2(s * n2, s * n2), p13, __fmul2_rn(make_float2(-s, -s), p7));
        fx = d.x;
        fz = d.y;
        return;
    }
    fx = pair_axis<false, kPotLJ>(n, c, inv43, dnx, h_coef, 0, 1.0f, 1.0f);
    fz = pair_axis<false, kPotLJ>(n, c, inv43, dnz, h_coef, 0, 1.0f, 1.0f);
}

// Pair energy of an atom (units D, twice the per-atom share: the caller halves it) in the x-z plane:
// cubic: the +-x and +-z pairs and the two y neighbours at rbar; HCP: the pairs above.
__device__ __forceinline__ float pair_energy_xz(float cr, float inv43, float dnx, float dnz, float h_coef, int pot_mode,
                                                float c_att, float s_rep, const EamP& eam = EamP{})
{
    if ((pot_mode & 3) == 3) {
        const float g[3] = {dnx, 0.0f, dnz};
        float F[3], u;
        eam_forces<2>(eam, cr * cr * cr, cr, inv43, g, h_coef, F, &u);
        return 2.0f * u;
    }
    if ((pot_mode & kLatHcp) == 0)
        return pair_energy_axis(cr, inv43, dnx, h_coef, pot_mode, c_att, s_rep) +
               pair_energy_axis(cr, inv43, dnz, h_coef, pot_mode, c_att, s_rep) + 2.0f * pair_U(pot_mode, c_att, s_rep, cr);
    return pair_energy_axis(cr, inv43, dnx, h_coef, pot_mode, c_att, s_rep) +
           2.0f * pair_energy_axis(cr, inv43, 0.5f * dnx, h_coef, pot_mode, c_att, s_rep) +
           pair_energy_axis(cr, inv43, 0.5f * dnx + kHcpS * dnz, h_coef, pot_mode, c_att, s_rep) +
           pair_energy_axis(cr, inv43, kHcpS * dnz, h_coef, pot_mode, c_att, s_rep) +
           pair_energy_axis(cr, inv43, -0.5f * dnx + kHcpS * dnz, h_coef, pot_mode, c_att, s_rep);
}

// 3D: the same lattices with the full gradient g. HCP pairs: basal (1, 0, 0), (1/2, h, 0),
// (-1/2, h, 0) with h = sqrt(3)/2 (weight 1), and the six out-of-plane directions
// (cos p / sqrt 3, sin p / sqrt 3, sqrt(2/3)), p = 30, 90, ..., 330 degrees, each paired with its
// opposite (weight 1/2: the two sublattices averaged).
constexpr float kHcpH = 0.866025403784439f;    // sqrt(3)/2
constexpr float kHcpR = 0.577350269189626f;    // 1/sqrt(3)

template <int POT = kPotRuntime>
__device__ __forceinline__ void pair_force3(float n, float c, float inv43, const float g[3], float h_coef, int pot_mode,
                                            float c_att, float s_rep, float F[3], const EamP& eam = EamP{})
{
    if ((POT >= 0 && (POT & 3) == kPotEam) || (POT == kPotRuntime && (pot_mode & 3) == 3)) {
        eam_forces<3>(eam, n, c, inv43, g, h_coef, F, nullptr);
        return;
    }
    const bool hcp = POT >= 0 ? (POT & kLatHcp) != 0 : (pot_mode & kLatHcp) != 0;
    if (!hcp) {
        for (int d = 0; d < 3; d++) F[d] = pair_axis<false, POT>(n, c, inv43, g[d], h_coef, pot_mode, c_att, s_rep);
        return;
    }
    const float b0 = pair_axis<false, POT>(n, c, inv43, g[0], h_coef, pot_mode, c_att, s_rep);
    const float b1 = pair_axis<false, POT>(n, c, inv43, 0.5f * g[0] + kHcpH * g[1], h_coef, pot_mode, c_att, s_rep);
    const float b2 = pair_axis<false, POT>(n, c, inv43, -0.5f * g[0] + kHcpH * g[1], h_coef, pot_mode, c_att, s_rep);
    F[0] = b0 + 0.5f * (b1 - b2);
    F[1] = kHcpH * (b1 + b2);
    F[2] = 0.0f;
    #pragma unroll
    for (int q = 0; q < 6; q++) {
        // cos and sin of 30 + 60 q degrees
        const float cq = q == 0 || q == 5 ? kHcpH : (q == 2 || q == 3 ? -kHcpH : 0.0f);
        const float sq = q == 1 ? 1.0f : (q == 4 ? -1.0f : (q == 0 || q == 2 ? 0.5f : -0.5f));
        const float ux = kHcpR * cq, uy = kHcpR * sq;
        const float a = 0.5f * pair_axis<false, POT>(n, c, inv43, ux * g[0] + uy * g[1] + kHcpS * g[2], h_coef,
                                                     pot_mode, c_att, s_rep);
        F[0] += a * ux;
        F[1] += a * uy;
        F[2] += a * kHcpS;
    }
}

// 3D pair energy (units D, twice the per-atom share).
__device__ __forceinline__ float pair_energy3(float cr, float inv43, const float g[3], float h_coef, int pot_mode,
                                             float c_att, float s_rep, const EamP& eam = EamP{})
{
    if ((pot_mode & 3) == 3) {
        float F[3], u;
        eam_forces<3>(eam, cr * cr * cr, cr, inv43, g, h_coef, F, &u);
        return 2.0f * u;
    }
    if ((pot_mode & kLatHcp) == 0) {
        float e = 0.0f;
        for (int d = 0; d < 3; d++) e += pair_energy_axis(cr, inv43, g[d], h_coef, pot_mode, c_att, s_rep);
        return e;
    }
    float e = pair_energy_axis(cr, inv43, g[0], h_coef, pot_mode, c_att, s_rep) +
              pair_energy_axis(cr, inv43, 0.5f * g[0] + kHcpH * g[1], h_coef, pot_mode, c_att, s_rep) +
              pair_energy_axis(cr, inv43, -0.5f * g[0] + kHcpH * g[1], h_coef, pot_mode, c_att, s_rep);
    for (int q = 0; q < 6; q++) {
        const float cq = q == 0 || q == 5 ? kHcpH : (q == 2 || q == 3 ? -kHcpH : 0.0f);
        const float sq = q == 1 ? 1.0f : (q == 4 ? -1.0f : (q == 0 || q == 2 ? 0.5f : -0.5f));
        e += 0.5f * pair_energy_axis(cr, inv43, kHcpR * (cq * g[0] + sq * g[1]) + kHcpS * g[2], h_coef, pot_mode,
                                     c_att, s_rep);
    }
    return e;
}

}  // namespace gbpic
