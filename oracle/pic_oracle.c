/*
 * pic_oracle.c -- plain FP64 CPU oracle of one particle-in-cell (PIC) cycle with the
 * pair-potential force of Mitchell, Schumacher & Chowdhury, "Modeling crater formation in
 * femtosecond-pulse laser damage from basic principles" (arXiv:1502.07722).
 *
 * TEST INFRASTRUCTURE. This library exists only to check the CUDA path. Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it. It shares no source,
 * header, table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * It is deliberately slow and literal: one particle at a time, one node at a time, FP64
 * throughout, no blocking, no fusion. Each function names the passage it follows.
 *
 * The cycle (paper, the PIC-cycle paragraph and Fig. 1):
 *   1. macroparticle weights are interpolated to the nearest surrounding nodes -> node density
 *   2. node density and its gradient at the half nodes are interpolated back to each
 *      macroparticle; the local environment gives nearest-neighbour distances (Eqs. 1-2) and
 *      the Lennard-Jones force (Eq. 3)
 *   3. Lorentz push (+ pair force), current deposition, Maxwell (Yee) field update.
 *
 * Readings where the paper is silent (all listed in the design notes of the repository):
 *   - the nodes nearest a particle: linear (cloud-in-cell) weights onto the 2 x 2 cell corners.
 *     Weights are fixed point: a coordinate X = rint(x * 2^16) (x in cell units), node weight
 *     S_j(X) = max(0, 2^16 - |X - 2^16 j|). Node sums are exact integers.
 *   - the gradient at the half nodes is the edge difference of the node density, interpolated
 *     linearly along the other axis; together with the bilinear node density this is the exact
 *     gradient of the interpolated density, hence consistent with the deposit.
 *   - densities are used in units of n0 = r0^-3, so rbar/r0 = (n/n0)^(-1/3).
 *   - Eq. (2): the neighbour on the +x side sits at rbar / (1 - g/2), the one on the -x side at
 *     rbar / (1 + g/2), g = d rbar / dx; a non-positive denominator puts that neighbour at
 *     infinity (no force). The force on the atom along x is U'(dr+) - U'(dr-).
 *   - In 2D the +-y neighbours sit at rbar (no force, counted in the energy).
 *   - Walls at z = 0 and z = nz reflect particles; the pair density on the wall node rows is
 *     doubled (mirror image of the slab behind the wall). x is periodic.
 *   - current deposition (not described in the paper) is Esirkepov's charge-conserving scheme
 *     for linear weights, evaluated in the same fixed point; J_y uses the code
 *     V = rint(beta_y * 2^b) taken in FP32 exactly as the kernel takes it, b = 18 unless the
 *     slab's particles per cell could overflow the int64 J_y node sums at that resolution
 *     (jy_bits below).
 *   - push: relativistic Boris with u = gamma v / c at half steps; the pair force is added to
 *     both half electric kicks.
 *   - fields: 2D3V Yee, B advanced in two half steps around the E update, first-order Mur at
 *     z = 0 and z = nz, laser launched by a J_x current sheet two node rows below the top.
 *   - variants the paper names as compatible: the Morse potential (pot_mode 2, minimum -D at r0)
 *     and the hexagonal close-packed lattice (lattice 1: Eq. 2 along each neighbour direction,
 *     ideal axial ratio, c axis along z, both sublattices' out-of-plane neighbours at weight 1/2).
 *   - the crater (Eq. 5's diameter, measured from the density map): material missing from each
 *     node column of the original slab, exact integer column sums times one factor (2D and 3D).
 * Every function is pinned by the tests against closed forms, invariants or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
#define O_C     299792458.0
#define O_QE    1.602176634e-19
#define O_ME    9.1093837015e-31
#define O_EPS0  8.8541878128e-12
#define O_KB    1.380649e-23
#define O_AMU   1.66053906660e-27
#define O_PI    3.14159265358979323846

#define QS 65536LL          /* fixed-point units per cell along one axis (2^16) */

/* ---------------------------------------------------------------------------------------- */
/* configuration: physical inputs                                                            */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t nx, nz;          /* cells along x (periodic) and z (walls)                       */
    int32_t slab_k;          /* the copper slab fills cell rows k < slab_k                    */
    int32_t mode;            /* 0: ions + electrons + fields; 1: neutral atoms only           */
    int32_t ppc_ion, ppc_electron;
    int32_t pot_mode;        /* 0: Eq. (3) as printed; 1: altered L-J (scaled branches); 2: Morse;
                                3: embedded-atom form (cubic lattice)                            */
    int32_t laser_profile;   /* 0: none; 1: plane wave; 2: focused Gaussian beam              */
    double dx;               /* cell size (m), square cells                                   */
    double cfl;              /* dt = cfl * dx / (c * sqrt(2)) when dt_override <= 0          */
    double dt_override;      /* s                                                             */
    double n_atoms;          /* solid density (m^-3)                                          */
    double T_ion_K, T_electron_eV;
    double ion_charge;       /* in units of e                                                 */
    double ion_mass_amu;
    double D_eV;             /* dissociation energy of Eq. (3)                                */
    double r0;               /* equilibrium distance of Eq. (3) (m); <= 0 -> n_atoms^(-1/3)  */
    double c_att, s_rep;     /* altered potential: factor on the attractive / repulsive side */
    double lambda, I0, tau_fwhm, w0, t_peak;   /* laser (m, W/m^2, s, m, s)                  */
    uint64_t seed;
    int32_t temp_profile;    /* 0: uniform T_ion_K; 1: lattice temperature of a laser spot       */
    int32_t lattice;         /* 0: cubic (the paper's); 1: hexagonal close-packed, c axis along z */
    double T_spot_K, spot_w, spot_depth;       /* K, m (1/e^2 radius), m (1/e depth)         */
    double morse_a;          /* Morse stiffness alpha r0 (pot_mode 2)                           */
    double eam_ec, eam_phi;  /* embedded-atom form (pot_mode 3): cohesive energy E_c and pair scale
                                phi_e (eV)                                                          */
    double eam_alpha, eam_beta, eam_gamma;   /* its exponents (dimensionless, r in units of r0)  */
} ocfg;

typedef struct {
    ocfg c;
    double dt, w, r0, D, rho_scale;     /* rho_scale: integer node sum -> n / n0           */
    int nsp;
    double q[2], m[2], uth[2];
    int pair[2];                        /* species that carries the pair force / density    */
    int64_t np[2];
    double *x[2], *z[2], *ux[2], *uy[2], *uz[2];
    double *F[6];                       /* Ex Ey Ez Bx By Bz, each (nz+1)*nx, row-major k,i */
    int64_t *rho;                       /* pair-species node sums at the current positions  */
    int64_t *J[3];                      /* J2x (i+1/2,k), J6y (i,k), J2z (i,k+1/2)           */
    int64_t step;
    /* laser */
    double E0, omega, kwave, t_ant, w_ant, R_ant, gouy_ant, amp_ant;
    int k_ant;
    double injected;                    /* field energy that crossed the row below the antenna
                                           towards the slab (J per metre of y)               */
    int32_t jy_bits;                    /* resolution of the J_y code (oracle_jy_bits)        */
} ostate;

static int64_t imod(int64_t a, int64_t n) { int64_t r = a % n; return r < 0 ? r + n : r; }
static int64_t floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b) != 0 && ((a < 0) != (b < 0))) q--; return q; }
static int64_t hat(int64_t X, int64_t j) { int64_t d = X - QS * j; if (d < 0) d = -d; return d < QS ? QS - d : 0; }
#define NODE(s, i, k) ((size_t)(k) * (size_t)(s)->c.nx + (size_t)(i))

/* ---------------------------------------------------------------------------------------- */
/* seeded generator for the initial state: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),   */
/* used counter-style: draw(key) = first output of a SplitMix64 generator seeded with        */
/* seed ^ key.                                                                               */
/* ---------------------------------------------------------------------------------------- */
static uint64_t splitmix64_first(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* key = ((species * 2^40 + particle) * 8 + draw) */
static uint64_t draw_bits(uint64_t seed, int s, uint64_t pidx, int d)
{
    uint64_t key = ((((uint64_t)s << 40) + pidx) << 3) + (uint64_t)d;
    return splitmix64_first(seed ^ key);
}
static double draw_unit24(uint64_t b) { return (double)(b >> 40) * (1.0 / 16777216.0); }      /* [0,1) */
static double draw_open53(uint64_t b) { return ((double)(b >> 11) + 1.0) * (1.0 / 9007199254740992.0); } /* (0,1] */

/* ---------------------------------------------------------------------------------------- */
/* Lennard-Jones pair potential, Eq. (3), in units of D with r in units of r0               */
/* ---------------------------------------------------------------------------------------- */
double oracle_lj_U(double r) { return pow(r, -12.0) - 2.0 * pow(r, -6.0); }
/* dU/dr (units D / r0) */
double oracle_lj_dU(double r) { return -12.0 * pow(r, -13.0) + 12.0 * pow(r, -7.0); }

/* branch factors of the altered potential (a finite stand-in for "infinite below r0" and the
 * multiplicative correction on the attractive side); plain Eq. (3) when pot_mode == 0 */
static double branch_factor_p(int pot_mode, double c_att, double s_rep, double r)
{
    if (pot_mode == 0) return 1.0;
    return r < 1.0 ? s_rep : c_att;
}
/* Morse potential (pot_mode 2; the paper names it as one the density-to-distance mapping takes
 * as it is), units of D with r in units of r0 and its minimum -1 at r = 1 like Eq. (3):
 * U = e^(-2 a (r - 1)) - 2 e^(-a (r - 1)), a = alpha r0 */
double oracle_morse_U(double a, double r) { double e = exp(-a * (r - 1.0)); return e * e - 2.0 * e; }
/* dU/dr (units D / r0) */
double oracle_morse_dU(double a, double r) { double e = exp(-a * (r - 1.0)); return 2.0 * a * e * (1.0 - e); }

/* the pair potential and its derivative selected by pot_mode */
static double pot_U(int pm, double c_att, double s_rep, double a, double r)
{
    return pm == 2 ? oracle_morse_U(a, r) : branch_factor_p(pm, c_att, s_rep, r) * oracle_lj_U(r);
}
static double pot_dU(int pm, double c_att, double s_rep, double a, double r)
{
    return pm == 2 ? oracle_morse_dU(a, r) : branch_factor_p(pm, c_att, s_rep, r) * oracle_lj_dU(r);
}

/* Eq. (1)-(2): nearest-neighbour distances (units r0) along one axis from the local density
 * n (units n0) and its derivative dn (units n0 per cell); r0_dx = r0 / dx.
 * Returns rbar; *plus / *minus are the distances to the neighbours on the + and - side
 * (INFINITY when the neighbour is pushed to infinity). */
double oracle_neighbor_distances(double n, double dn, double r0_dx, double* plus, double* minus)
{
    double rbar = pow(n, -1.0 / 3.0);                                 /* rbar = n^(-1/3)    */
    double g = -(1.0 / 3.0) * dn * pow(n, -4.0 / 3.0) * r0_dx;        /* Eq. (1)            */
    double dp = 1.0 - 0.5 * g, dm = 1.0 + 0.5 * g;                    /* Eq. (2)            */
    *plus = dp > 0.0 ? rbar / dp : INFINITY;
    *minus = dm > 0.0 ? rbar / dm : INFINITY;
    return rbar;
}

/* Nearest-neighbour directions (unit vectors) and weights of the lattice the atoms are assumed
 * to form (paper: a cubic lattice, readily replaced by a hexagonal close-packed one).
 * Cubic: the six axis directions, weight 1. HCP with the ideal axial ratio and the c axis along z:
 * six neighbours in the basal plane at 60-degree steps from +x (weight 1), and three above and
 * three below the plane at in-plane radius 1/sqrt(3) and height sqrt(2/3); the two sublattices
 * place those triples 60 degrees apart and a density field cannot tell them apart, so both
 * sublattices' twelve out-of-plane directions enter with weight 1/2. Returns the count. */
static int lattice_dirs(int lattice, double e[18][3], double w[18])
{
    int m = 0;
    if (lattice == 0) {
        for (int d = 0; d < 3; d++)
            for (int sg = -1; sg <= 1; sg += 2) {
                e[m][0] = e[m][1] = e[m][2] = 0.0;
                e[m][d] = sg;
                w[m++] = 1.0;
            }
        return m;
    }
    for (int q = 0; q < 6; q++) {
        double th = q * O_PI / 3.0;
        e[m][0] = cos(th); e[m][1] = sin(th); e[m][2] = 0.0; w[m++] = 1.0;
    }
    double rin = 1.0 / sqrt(3.0), h = sqrt(2.0 / 3.0);
    for (int q = 0; q < 6; q++) {                    /* phi = 30, 90, ..., 330 degrees */
        double ph = O_PI / 6.0 + q * O_PI / 3.0;
        for (int sg = -1; sg <= 1; sg += 2) {
            e[m][0] = rin * cos(ph); e[m][1] = rin * sin(ph); e[m][2] = sg * h; w[m++] = 0.5;
        }
    }
    return m;
}

/* Pair force (units D / r0, per axis) and energy (units D, half the sum of U) of an atom at local
 * density n (units n0) with density gradient grad (units n0 per cell) on a lattice of directions
 * e_k: each neighbour sits where Eq. (2), taken along e_k, puts it (rbar over 1 - (grad rbar . e_k)
 * / 2, from Eq. 1 along e_k), and the force is the sum of w_k U'(r_k) e_k. */
static void lattice_pair(int lattice, int pm, double ca, double sr, double ma, double n, const double grad[3],
                         double r0_dx, double F[3], double* u)
{
    double e[18][3], w[18];
    int m = lattice_dirs(lattice, e, w);
    F[0] = F[1] = F[2] = 0.0;
    *u = 0.0;
    for (int k = 0; k < m; k++) {
        double dn = e[k][0] * grad[0] + e[k][1] * grad[1] + e[k][2] * grad[2];
        double rk, unused;
        oracle_neighbor_distances(n, dn, r0_dx, &rk, &unused);
        if (isinf(rk)) continue;
        double du = w[k] * pot_dU(pm, ca, sr, ma, rk);
        for (int d = 0; d < 3; d++) F[d] += du * e[k][d];
        *u += 0.5 * w[k] * pot_U(pm, ca, sr, ma, rk);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* embedded-atom form (pot_mode 3): the paper notes that other potentials are readily adapted  */
/* to its mapping of density to neighbour distance. The analytic nearest-neighbour EAM of      */
/* Johnson (Phys. Rev. B 37, 3924, 1988), rebuilt for the paper's cubic lattice of six        */
/* nearest neighbours, with r in units of r0 (the equilibrium spacing) and energies in units  */
/* of D:                                                                                       */
/*   electron density of one neighbour  f(r)   = exp(-beta (r - 1))                            */
/*   pair term                          phi(r) = phi_e exp(-gamma (r - 1))                     */
/*   embedding energy                   F(rho) = -E_c (1 - (alpha/beta) ln x) x^(alpha/beta)   */
/*                                               - 3 phi_e x^(gamma/beta),  x = rho / 6        */
/* so that a uniform lattice of spacing r has E = F(6 f(r)) + 3 phi(r) = -E_c (1 + a) e^(-a),  */
/* a = alpha (r - 1) (the universal binding curve), -E_c at r = 1.                             */
/* Reading of the one-atom environment: atom i's embedding density is the sum of f over its   */
/* six Eq. (2) neighbours (+-y at rbar in 2D); neighbour j's own embedding density is          */
/* 6 f(rbar_j) with rbar_j = n_j^(-1/3) and n_j the interpolated density at j's position, taken */
/* along the axis from the atom's density and its gradient (n + s dn, s the neighbour's offset */
/* in cells), but never less than f(r), the density of its own bond back to the atom (any     */
/* neighbour holds that bond; in a steep gradient, as at a free surface, n_j can fall towards  */
/* zero, where F'(rho) diverges like rho^(alpha/beta - 1) ln rho); the bond to j pulls with    */
/* T = phi'(r) + (F'(rho_i) + F'(rho_j)) f'(r), and the force along an axis is T(r+) - T(r-),  */
/* as U'(r+) - U'(r-) for a pair potential.                                                    */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    double ec, phi, alpha, beta, gamma;      /* ec, phi in units of D */
} eam_p;

static double eam_f(const eam_p* p, double r) { return exp(-p->beta * (r - 1.0)); }
static double eam_df(const eam_p* p, double r) { return -p->beta * exp(-p->beta * (r - 1.0)); }
static double eam_phi(const eam_p* p, double r) { return p->phi * exp(-p->gamma * (r - 1.0)); }
static double eam_dphi(const eam_p* p, double r) { return -p->gamma * p->phi * exp(-p->gamma * (r - 1.0)); }
static double eam_F(const eam_p* p, double rho)
{
    if (!(rho > 0.0)) return 0.0;
    double x = rho / 6.0, k = p->alpha / p->beta, m = p->gamma / p->beta;
    return -p->ec * (1.0 - k * log(x)) * pow(x, k) - 3.0 * p->phi * pow(x, m);
}
static double eam_dF(const eam_p* p, double rho)          /* dF / d rho */
{
    if (!(rho > 0.0)) return 0.0;
    double x = rho / 6.0, k = p->alpha / p->beta, m = p->gamma / p->beta;
    return (p->ec * k * k * log(x) * pow(x, k - 1.0) - 3.0 * p->phi * m * pow(x, m - 1.0)) / 6.0;
}

/* Force (units D / r0) and energy (units D) of an atom at density n with gradient grad (n0 per
 * cell) under the embedded-atom form; axes: 2 (x and z, the y neighbours at rbar) or 3. */
static void eam_atom(const eam_p* p, double n, const double grad[3], int three_d, double r0_dx, double F[3],
                     double* u)
{
    double rp[3], rm[3];
    double rbar = pow(n, -1.0 / 3.0), rho = 0.0, upair = 0.0;
    F[0] = F[1] = F[2] = 0.0;
    for (int d = 0; d < 3; d++) {
        if (!three_d && d == 1) {                 /* 2D: the +-y neighbours at rbar */
            rp[d] = rm[d] = rbar;
        } else {
            oracle_neighbor_distances(n, grad[d], r0_dx, &rp[d], &rm[d]);
        }
        if (!isinf(rp[d])) { rho += eam_f(p, rp[d]); upair += eam_phi(p, rp[d]); }
        if (!isinf(rm[d])) { rho += eam_f(p, rm[d]); upair += eam_phi(p, rm[d]); }
    }
    double dFi = eam_dF(p, rho);
    for (int d = 0; d < 3; d++) {
        if (!three_d && d == 1) continue;
        double T[2] = {0.0, 0.0};
        for (int side = 0; side < 2; side++) {
            double r = side == 0 ? rp[d] : rm[d];
            if (isinf(r)) continue;
            double nj = n + (side == 0 ? 1.0 : -1.0) * r * r0_dx * grad[d];
            double rhoj = nj > 0.0 ? 6.0 * eam_f(p, pow(nj, -1.0 / 3.0)) : 0.0;
            if (rhoj < eam_f(p, r)) rhoj = eam_f(p, r);     /* at least the bond back to the atom */
            double dFj = eam_dF(p, rhoj);
            T[side] = eam_dphi(p, r) + (dFi + dFj) * eam_df(p, r);
        }
        F[d] = T[0] - T[1];
    }
    *u = eam_F(p, rho) + 0.5 * upair;
}

/* the form's parameters in units of D */
static eam_p eam_params(double D_eV, double ec, double phi, double alpha, double beta, double gamma)
{
    eam_p p = {ec / D_eV, phi / D_eV, alpha, beta, gamma};
    return p;
}

/* Force (units D / r0) and energy (units D) on an atom at density n, gradient dnx, dnz (2D), for
 * the probes of the tests */
void oracle_eam_atom2(double D_eV, double ec, double phi, double alpha, double beta, double gamma, double n,
                      double dnx, double dnz, double r0_dx, double out[3])
{
    eam_p p = eam_params(D_eV, ec, phi, alpha, beta, gamma);
    double grad[3] = {dnx, 0.0, dnz}, F[3], u;
    if (!(n > 0.0)) { out[0] = out[1] = out[2] = 0.0; return; }
    eam_atom(&p, n, grad, 0, r0_dx, F, &u);
    out[0] = F[0];
    out[1] = F[2];
    out[2] = u;
}

/* ---------------------------------------------------------------------------------------- */
/* node density (pair species), paper's PIC-cycle paragraph: weights to the nearest nodes   */
/* ---------------------------------------------------------------------------------------- */
static void deposit_density_one(int nx, int nz, int64_t* rho, double x, double z)
{
    int64_t X = llrint(x * (double)QS), Z = llrint(z * (double)QS);
    int64_t j0 = floordiv(X, QS), l0 = floordiv(Z, QS);
    for (int64_t l = l0; l <= l0 + 1; l++) {
        int64_t sz = hat(Z, l);
        if (sz == 0) continue;
        for (int64_t j = j0; j <= j0 + 1; j++) {
            int64_t sx = hat(X, j);
            if (sx == 0) continue;
            if (l < 0 || l > nz) abort();
            rho[(size_t)l * nx + imod(j, nx)] += sx * sz;
        }
    }
}

void oracle_deposit_density(int32_t nx, int32_t nz, int64_t n, const double* x, const double* z, int64_t* rho)
{
    memset(rho, 0, sizeof(int64_t) * (size_t)nx * (size_t)(nz + 1));
    for (int64_t p = 0; p < n; p++) deposit_density_one(nx, nz, rho, x[p], z[p]);
}

/* ---------------------------------------------------------------------------------------- */
/* current deposition: Esirkepov (Comput. Phys. Commun. 135, 144 (2001)) for linear weights, */
/* in the fixed point of the density. Integer identities:                                   */
/*   2 Wx(j,l) = dSx(j) (S0z(l) + S1z(l))      2 Wz = dSz (S0x + S1x)                        */
/*   6 Wy(j,l) = 2 S0x S0z + S1x S0z + S0x S1z + 2 S1x S1z                                   */
/*   J2x(j+1/2,l) = J2x(j-1/2,l) - 2 Wx(j,l)   (and the same along z)                        */
/* so that 2 (rho1 - rho0) + div(J2) = 0 exactly.                                            */
/* V is the J_y code of the particle.                                                        */
/* ---------------------------------------------------------------------------------------- */
static void deposit_current_one(int nx, int nz, int64_t* J2x, int64_t* J6y, int64_t* J2z, int64_t sign,
                                int64_t X0, int64_t Z0, int64_t X1, int64_t Z1, int64_t V)
{
    int64_t bx = floordiv(X0 < X1 ? X0 : X1, QS), bz = floordiv(Z0 < Z1 ? Z0 : Z1, QS);
    int64_t S0x[3], S1x[3], S0z[3], S1z[3];
    for (int a = 0; a < 3; a++) {
        S0x[a] = hat(X0, bx + a); S1x[a] = hat(X1, bx + a);
        S0z[a] = hat(Z0, bz + a); S1z[a] = hat(Z1, bz + a);
    }
    /* both shapes must lie inside the 3-node window (a move of less than one cell) */
    int64_t t0 = 0, t1 = 0, u0 = 0, u1 = 0;
    for (int a = 0; a < 3; a++) { t0 += S0x[a]; t1 += S1x[a]; u0 += S0z[a]; u1 += S1z[a]; }
    if (t0 != QS || t1 != QS || u0 != QS || u1 != QS) abort();

    for (int b = 0; b < 3; b++) {            /* J_x along each node row */
        int64_t acc = 0;
        for (int a = 0; a < 2; a++) {
            acc -= (S1x[a] - S0x[a]) * (S0z[b] + S1z[b]);
            if (acc != 0) {
                int64_t l = bz + b;
                if (l < 0 || l > nz) abort();
                J2x[(size_t)l * nx + imod(bx + a, nx)] += sign * acc;
            }
        }
    }
    for (int a = 0; a < 3; a++) {            /* J_z along each node column */
        int64_t acc = 0;
        for (int b = 0; b < 2; b++) {
            acc -= (S1z[b] - S0z[b]) * (S0x[a] + S1x[a]);
            if (acc != 0) {
                int64_t l = bz + b;
                if (l < 0 || l > nz - 1) abort();
                J2z[(size_t)l * nx + imod(bx + a, nx)] += sign * acc;
            }
        }
    }
    if (V != 0) {
        for (int b = 0; b < 3; b++)
            for (int a = 0; a < 3; a++) {
                int64_t w6 = 2 * S0x[a] * S0z[b] + S1x[a] * S0z[b] + S0x[a] * S1z[b] + 2 * S1x[a] * S1z[b];
                if (w6 != 0) {
                    int64_t l = bz + b;
                    if (l < 0 || l > nz) abort();
                    J6y[(size_t)l * nx + imod(bx + a, nx)] += sign * V * w6;
                }
            }
    }
}

/* J_y code: V = rint(beta_y * 2^bits), beta_y = u_y / gamma, all in FP32 without fused
 * multiply-add, so that the decision is the kernel's (this file is built with contraction off).
 * The kernel's definition of 1/gamma: for u^2 < 2^-10 the series 1 - u^2 (1/2 - 3/8 u^2),
 * otherwise 1 / sqrt(1 + u^2). */
int64_t oracle_jy_code(float ux, float uy, float uz, int32_t bits)
{
    float u2 = ux * ux;
    u2 = u2 + uy * uy;
    u2 = u2 + uz * uz;
    float by;
    if (u2 < 0.0009765625f) {
        float t = u2 * 0.375f;
        t = 0.5f - t;
        t = u2 * t;
        by = uy * (1.0f - t);
    } else {
        float g = sqrtf(1.0f + u2);
        by = uy / g;
    }
    return (int64_t)rintf(by * ldexpf(1.0f, bits));
}

/* Resolution of the J_y code for a 2D slab with the given macroparticles per cell (both species).
 * One particle adds at most 2^bits * 6 * 2^32 to a J_y node sum (|beta_y| < 1; the six-fold
 * weight of a node is at most 6 * 2^32) and the particles that reach a node sit in a block of
 * 4 x 4 cells, so the int64 sum cannot overflow while such a block holds at most
 * floor(2^63 / (6 * 2^(32+bits))) particles. bits = 18, or the largest bits whose limit holds
 * 1.25 times the 16 * per_cell particles of a block of the initial slab. */
int32_t oracle_jy_bits(int64_t per_cell)
{
    for (int32_t b = 18; b >= 1; b--) {
        int64_t limit = (INT64_C(1) << 31) / (INT64_C(6) << b);
        if ((double)limit >= 1.25 * 16.0 * (double)per_cell) return b;
    }
    return 0;
}

/* Unwrap the new x coordinate (periodic, period nx) to within half a period of the old one. */
static int64_t unwrap_X(int64_t X0, int64_t X1, int nx)
{
    int64_t P = (int64_t)nx * QS;
    while (X1 - X0 > P / 2) X1 -= P;
    while (X0 - X1 > P / 2) X1 += P;
    return X1;
}

/* Deposit the current of n particles that moved from (x0,z0) to (x1,z1) with new momenta u
 * (FP32, the state the kernel stores). Accumulates into J2x, J6y, J2z. */
void oracle_deposit_current(int32_t nx, int32_t nz, int64_t n, int32_t sign,
                            const double* x0, const double* z0, const double* x1, const double* z1,
                            const float* ux, const float* uy, const float* uz, int32_t bits,
                            int64_t* J2x, int64_t* J6y, int64_t* J2z)
{
    for (int64_t p = 0; p < n; p++) {
        int64_t X0 = llrint(x0[p] * (double)QS), Z0 = llrint(z0[p] * (double)QS);
        int64_t X1 = unwrap_X(X0, llrint(x1[p] * (double)QS), nx), Z1 = llrint(z1[p] * (double)QS);
        deposit_current_one(nx, nz, J2x, J6y, J2z, sign, X0, Z0, X1, Z1, oracle_jy_code(ux[p], uy[p], uz[p], bits));
    }
}

/* ---------------------------------------------------------------------------------------- */
/* interpolation back to the particle                                                        */
/* ---------------------------------------------------------------------------------------- */
/* pair density at a node in units of n0; wall rows doubled (mirror image behind the wall) */
static double nhat_node(const ostate* s, int64_t i, int64_t k)
{
    double v = (double)s->rho[NODE(s, imod(i, s->c.nx), k)] * s->rho_scale;
    if (k == 0 || k == s->c.nz) v *= 2.0;
    return v;
}

/* bilinear node density and its gradient (per cell) at (x, z): the gradient is the edge
 * difference at the half nodes, interpolated along the other axis (paper: density gradient at
 * the half-node positions, interpolated back self-consistently) */
static void gather_density(const ostate* s, double x, double z, double* n, double* dn_dxi, double* dn_dzeta)
{
    int64_t i = (int64_t)floor(x), k = (int64_t)floor(z);
    double fx = x - (double)i, fz = z - (double)k;
    if (k >= s->c.nz) { k = s->c.nz - 1; fz = 1.0; }
    double n00 = nhat_node(s, i, k), n10 = nhat_node(s, i + 1, k);
    double n01 = nhat_node(s, i, k + 1), n11 = nhat_node(s, i + 1, k + 1);
    *n = (1 - fx) * (1 - fz) * n00 + fx * (1 - fz) * n10 + (1 - fx) * fz * n01 + fx * fz * n11;
    *dn_dxi = (1 - fz) * (n10 - n00) + fz * (n11 - n01);
    *dn_dzeta = (1 - fx) * (n01 - n00) + fx * (n11 - n10);
}

/* staggered bilinear gather of a Yee component located at (i + sx, k + sz) */
static double gather_field(const ostate* s, const double* A, double x, double z, double sx, double sz)
{
    int nx = s->c.nx, nz = s->c.nz;
    double xs = x - sx, zs = z - sz;
    int64_t rows = sz > 0 ? nz : nz + 1;      /* half-row components have nz rows */
    if (zs < 0.0) zs = 0.0;
    if (zs > (double)(rows - 1)) zs = (double)(rows - 1);
    int64_t i = (int64_t)floor(xs), k = (int64_t)floor(zs);
    double fx = xs - (double)i, fz = zs - (double)k;
    if (k >= rows - 1) { k = rows - 2; fz = 1.0; }
    int64_t i0 = imod(i, nx), i1 = imod(i + 1, nx);
    return (1 - fx) * (1 - fz) * A[(size_t)k * nx + i0] + fx * (1 - fz) * A[(size_t)k * nx + i1]
         + (1 - fx) * fz * A[(size_t)(k + 1) * nx + i0] + fx * fz * A[(size_t)(k + 1) * nx + i1];
}

/* Force (N, per atom) on an atom at (x, z) from the current node density, Eqs. (1)-(3).
 * If energy is not NULL it receives the atom's pair energy (J): half the sum of U over its
 * six nearest neighbours (+-x, +-z from Eq. 2, +-y at rbar). */
static void pair_force_at(const ostate* s, double x, double z, double F[3], double* energy)
{
    double n, dnx, dnz;
    gather_density(s, x, z, &n, &dnx, &dnz);
    F[0] = F[1] = F[2] = 0.0;
    if (energy) *energy = 0.0;
    if (!(n > 0.0)) return;
    double r0_dx = s->r0 / s->c.dx;
    if (s->c.pot_mode == 3) {
        eam_p p = eam_params(s->c.D_eV, s->c.eam_ec, s->c.eam_phi, s->c.eam_alpha, s->c.eam_beta, s->c.eam_gamma);
        double grad[3] = {dnx, 0.0, dnz}, Fu[3], u;
        eam_atom(&p, n, grad, 0, r0_dx, Fu, &u);
        for (int d = 0; d < 3; d++) F[d] = (s->D / s->r0) * Fu[d];
        if (energy) *energy = s->D * u;
        return;
    }
    if (s->c.lattice == 1) {
        double grad[3] = {dnx, 0.0, dnz}, Fu[3], u;
        lattice_pair(1, s->c.pot_mode, s->c.c_att, s->c.s_rep, s->c.morse_a, n, grad, r0_dx, Fu, &u);
        for (int d = 0; d < 3; d++) F[d] = (s->D / s->r0) * Fu[d];
        if (energy) *energy = s->D * u;
        return;
    }
    double ap, am, bp, bm;
    double rbar = oracle_neighbor_distances(n, dnx, r0_dx, &ap, &am);
    oracle_neighbor_distances(n, dnz, r0_dx, &bp, &bm);
    double f_unit = s->D / s->r0;
    int pm = s->c.pot_mode;
    double ca = s->c.c_att, sr = s->c.s_rep, ma = s->c.morse_a;
    double dUap = isinf(ap) ? 0.0 : pot_dU(pm, ca, sr, ma, ap);
    double dUam = isinf(am) ? 0.0 : pot_dU(pm, ca, sr, ma, am);
    double dUbp = isinf(bp) ? 0.0 : pot_dU(pm, ca, sr, ma, bp);
    double dUbm = isinf(bm) ? 0.0 : pot_dU(pm, ca, sr, ma, bm);
    F[0] = f_unit * (dUap - dUam);
    F[2] = f_unit * (dUbp - dUbm);
    if (energy) {
        double u = 0.0;
        if (!isinf(ap)) u += pot_U(pm, ca, sr, ma, ap);
        if (!isinf(am)) u += pot_U(pm, ca, sr, ma, am);
        if (!isinf(bp)) u += pot_U(pm, ca, sr, ma, bp);
        if (!isinf(bm)) u += pot_U(pm, ca, sr, ma, bm);
        u += 2.0 * pot_U(pm, ca, sr, ma, rbar);
        *energy = 0.5 * s->D * u;
    }
}

/* ---------------------------------------------------------------------------------------- */
/* relativistic Boris push (u = gamma v / c), pair force added to both half kicks            */
/* ---------------------------------------------------------------------------------------- */
void oracle_boris(double q, double m, double dt, const double E[3], const double B[3], const double Fp[3], double u[3])
{
    double eps = q * dt / (2.0 * m * O_C);          /* electric half kick per (V/m)          */
    double fk = dt / (2.0 * m * O_C);               /* pair-force half kick per N             */
    double um[3], up[3], t[3], sv[3], uprime[3];
    for (int d = 0; d < 3; d++) um[d] = u[d] + eps * E[d] + fk * Fp[d];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double tfac = q * dt / (2.0 * m * gm);
    for (int d = 0; d < 3; d++) t[d] = tfac * B[d];
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int d = 0; d < 3; d++) sv[d] = 2.0 * t[d] / (1.0 + t2);
    uprime[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    uprime[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    uprime[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    up[0] = um[0] + (uprime[1] * sv[2] - uprime[2] * sv[1]);
    up[1] = um[1] + (uprime[2] * sv[0] - uprime[0] * sv[2]);
    up[2] = um[2] + (uprime[0] * sv[1] - uprime[1] * sv[0]);
    for (int d = 0; d < 3; d++) u[d] = up[d] + eps * E[d] + fk * Fp[d];
}

/* ---------------------------------------------------------------------------------------- */
/* laser source: E_x of the incident pulse at the antenna row                                */
/* ---------------------------------------------------------------------------------------- */
static double laser_field(const ostate* s, double x_cells, double t)
{
    if (s->c.laser_profile == 0) return 0.0;
    double tau = t - s->t_ant;
    double env = exp(-2.0 * log(2.0) * tau * tau / (s->c.tau_fwhm * s->c.tau_fwhm));
    if (s->c.laser_profile == 1) return s->E0 * env * sin(s->omega * tau);
    double xr = (x_cells - 0.5 * s->c.nx) * s->c.dx;
    double amp = s->amp_ant * exp(-xr * xr / (s->w_ant * s->w_ant));
    double phase = -s->kwave * xr * xr / (2.0 * s->R_ant) + s->gouy_ant;
    return s->E0 * amp * env * sin(s->omega * tau + phase);
}

/* ---------------------------------------------------------------------------------------- */
/* Maxwell, 2D3V Yee (d/dy = 0). Ex(i+1/2,k) Ey(i,k) Ez(i,k+1/2) Bx(i,k+1/2) By(i+1/2,k+1/2)  */
/* Bz(i+1/2,k); node rows k = 0..nz, half rows k = 0..nz-1                                   */
/* ---------------------------------------------------------------------------------------- */
static void half_step_B(ostate* s)
{
    int nx = s->c.nx, nz = s->c.nz;
    double h = 0.5 * s->dt / s->c.dx;
    double *Ex = s->F[0], *Ey = s->F[1], *Ez = s->F[2], *Bx = s->F[3], *By = s->F[4], *Bz = s->F[5];
    for (int k = 0; k <= nz; k++)
        for (int i = 0; i < nx; i++) {
            int ip = (i + 1) % nx;
            if (k < nz) {
                /* dBx/dt = dEy/dz ; dBy/dt = dEz/dx - dEx/dz */
                Bx[NODE(s, i, k)] += h * (Ey[NODE(s, i, k + 1)] - Ey[NODE(s, i, k)]);
                By[NODE(s, i, k)] += h * ((Ez[NODE(s, ip, k)] - Ez[NODE(s, i, k)]) - (Ex[NODE(s, i, k + 1)] - Ex[NODE(s, i, k)]));
            }
            /* dBz/dt = -dEy/dx */
            Bz[NODE(s, i, k)] -= h * (Ey[NODE(s, ip, k)] - Ey[NODE(s, i, k)]);
        }
}

static void full_step_E(ostate* s)
{
    int nx = s->c.nx, nz = s->c.nz;
    double cdt = O_C * s->dt, h = O_C * O_C * s->dt / s->c.dx;
    double *Ex = s->F[0], *Ey = s->F[1], *Ez = s->F[2], *Bx = s->F[3], *By = s->F[4], *Bz = s->F[5];
    size_t nn = (size_t)nx * (nz + 1);
    double* nEx = malloc(sizeof(double) * nn);
    double* nEy = malloc(sizeof(double) * nn);
    /* J (integer) -> dt J / eps0 */
    double cjx = O_QE * s->w / (8589934592.0 * s->c.dx * O_EPS0);                 /* 2^33 */
    double cjy = O_QE * s->w * O_C * s->dt / (6.0 * ldexp(1.0, 32 + s->jy_bits) * s->c.dx * s->c.dx * O_EPS0);
    double tmid = ((double)s->step + 0.5) * s->dt;
    for (int k = 0; k <= nz; k++)
        for (int i = 0; i < nx; i++) {
            int im = (i + nx - 1) % nx;
            size_t c = NODE(s, i, k);
            nEx[c] = Ex[c];
            nEy[c] = Ey[c];
            if (k > 0 && k < nz) {
                /* dEx/dt = -c^2 dBy/dz - Jx/eps0 ; dEy/dt = c^2 (dBx/dz - dBz/dx) - Jy/eps0 */
                nEx[c] = Ex[c] - h * (By[c] - By[NODE(s, i, k - 1)]) - cjx * (double)s->J[0][c];
                nEy[c] = Ey[c] + h * ((Bx[c] - Bx[NODE(s, i, k - 1)]) - (Bz[c] - Bz[NODE(s, im, k)])) - cjy * (double)s->J[1][c];
                if (k == s->k_ant) nEx[c] += 2.0 * (cdt / s->c.dx) * laser_field(s, (double)i + 0.5, tmid);
            }
        }
    /* first-order Mur on the wall rows for the tangential components */
    double alpha = (cdt - s->c.dx) / (cdt + s->c.dx);
    for (int i = 0; i < nx; i++) {
        size_t b0 = NODE(s, i, 0), b1 = NODE(s, i, 1), t0 = NODE(s, i, nz), t1 = NODE(s, i, nz - 1);
        nEx[b0] = Ex[b1] + alpha * (nEx[b1] - Ex[b0]);
        nEy[b0] = Ey[b1] + alpha * (nEy[b1] - Ey[b0]);
        nEx[t0] = Ex[t1] + alpha * (nEx[t1] - Ex[t0]);
        nEy[t0] = Ey[t1] + alpha * (nEy[t1] - Ey[t0]);
    }
    for (int k = 0; k < nz; k++)
        for (int i = 0; i < nx; i++) {
            int ip = (i + 1) % nx;
            size_t c = NODE(s, i, k);
            /* dEz/dt = c^2 dBy/dx - Jz/eps0 */
            Ez[c] += h * (By[c] - By[NODE(s, (i + nx - 1) % nx, k)]) - cjx * (double)s->J[2][c];
            (void)ip;
        }
    /* injected energy: Poynting flux S_z = (Ex By - Ey Bx) / mu0 through the node row below the
     * antenna, E at the half step (mean of old and new), B at the half step, B averaged over the
     * half rows on either side; energy moving towards the slab (-z) counts positive */
    int kp = s->k_ant - 1;
    if (kp >= 1 && kp < nz) {
        double mu0 = 1.0 / (O_EPS0 * O_C * O_C), sum = 0.0;
        for (int i = 0; i < nx; i++) {
            size_t c = NODE(s, i, kp), d = NODE(s, i, kp - 1);
            double ex = 0.5 * (Ex[c] + nEx[c]), ey = 0.5 * (Ey[c] + nEy[c]);
            sum += ex * 0.5 * (By[d] + By[c]) - ey * 0.5 * (Bx[d] + Bx[c]);
        }
        s->injected -= sum / mu0 * s->c.dx * s->dt;
    }
    memcpy(Ex, nEx, sizeof(double) * nn);
    memcpy(Ey, nEy, sizeof(double) * nn);
    free(nEx); free(nEy);
}

double oracle_injected(const ostate* s) { return s->injected; }

/* ---------------------------------------------------------------------------------------- */
/* state management                                                                          */
/* ---------------------------------------------------------------------------------------- */
static void redeposit(ostate* s)
{
    oracle_deposit_density(s->c.nx, s->c.nz, s->np[0], s->x[0], s->z[0], s->rho);
}

static void alloc_species(ostate* s, int sp, int64_t n)
{
    free(s->x[sp]); free(s->z[sp]); free(s->ux[sp]); free(s->uy[sp]); free(s->uz[sp]);
    s->np[sp] = n;
    size_t b = sizeof(double) * (size_t)(n > 0 ? n : 1);
    s->x[sp] = calloc(1, b); s->z[sp] = calloc(1, b);
    s->ux[sp] = calloc(1, b); s->uy[sp] = calloc(1, b); s->uz[sp] = calloc(1, b);
}

/* Initial state (paper: a damage simulation is initialised for target density and
 * temperature): a slab of cell rows k < slab_k, ppc macro-ions per cell at uniformly drawn
 * positions, Maxwellian momenta; electrons co-located with the ions (zero net charge, E = 0). */
/* Lattice temperature the atomic-transport run starts from (paper: initialisation paragraph and
 * Fig. 2, the lattice temperature once electrons and lattice have equilibrated; the figure itself
 * is not available, so a synthetic laser spot stands in for it): at the surface row slab_k the
 * temperature rises from T_ion_K to T_spot_K on the axis x = nx/2 with a Gaussian of 1/e^2
 * radius spot_w, and decays into the slab with 1/e depth spot_depth. (x, z) in cells. */
static double spot_temperature(const ocfg* c, double x, double z)
{
    double lateral = (x - 0.5 * c->nx) * c->dx / c->spot_w;
    double depth = (c->slab_k - z) * c->dx / c->spot_depth;
    return c->T_ion_K + (c->T_spot_K - c->T_ion_K) * exp(-2.0 * lateral * lateral) * exp(-depth);
}

/* initial state of the particle in slot j of cell (i, k) of species sp: x, z, ux, uy, uz */
static void init_one(const ostate* s, int sp, int64_t i, int64_t k, int64_t j, double out[5])
{
    const ocfg* c = &s->c;
    int ppc = sp == 0 ? c->ppc_ion : c->ppc_electron;
    uint64_t cellidx = (uint64_t)k * (uint64_t)c->nx + (uint64_t)i;
    /* positions: electrons reuse the ion draws of the same (cell, slot) */
    int pos_sp = (sp == 1 && c->ppc_electron == c->ppc_ion) ? 0 : sp;
    uint64_t pid_pos = cellidx * (uint64_t)ppc + (uint64_t)j;
    out[0] = (double)i + draw_unit24(draw_bits(c->seed, pos_sp, pid_pos, 0));
    out[1] = (double)k + draw_unit24(draw_bits(c->seed, pos_sp, pid_pos, 1));
    /* Box-Muller normals from two pairs of draws */
    double r1 = sqrt(-2.0 * log(draw_open53(draw_bits(c->seed, sp, pid_pos, 2))));
    double a1 = 2.0 * O_PI * draw_unit24(draw_bits(c->seed, sp, pid_pos, 3));
    double r2 = sqrt(-2.0 * log(draw_open53(draw_bits(c->seed, sp, pid_pos, 4))));
    double a2 = 2.0 * O_PI * draw_unit24(draw_bits(c->seed, sp, pid_pos, 5));
    double uth = s->uth[sp];
    if (sp == 0 && c->temp_profile == 1)
        uth = sqrt(O_KB * spot_temperature(c, out[0], out[1]) / (s->m[0] * O_C * O_C));
    out[2] = uth * r1 * cos(a1);
    out[3] = uth * r1 * sin(a1);
    out[4] = uth * r2 * cos(a2);
}

static void init_particles(ostate* s)
{
    const ocfg* c = &s->c;
    int64_t ncell = (int64_t)c->nx * c->slab_k;
    for (int sp = 0; sp < s->nsp; sp++) {
        int ppc = sp == 0 ? c->ppc_ion : c->ppc_electron;
        alloc_species(s, sp, ncell * ppc);
        int64_t p = 0;
        for (int k = 0; k < c->slab_k; k++)
            for (int i = 0; i < c->nx; i++)
                for (int j = 0; j < ppc; j++, p++) {
                    double v[5];
                    init_one(s, sp, i, k, j, v);
                    s->x[sp][p] = v[0]; s->z[sp][p] = v[1];
                    s->ux[sp][p] = v[2]; s->uy[sp][p] = v[3]; s->uz[sp][p] = v[4];
                }
    }
}

ostate* oracle_create(const ocfg* cfg, int32_t with_particles)
{
    ostate* s = calloc(1, sizeof(ostate));
    s->c = *cfg;
    const ocfg* c = &s->c;
    s->dt = c->dt_override > 0 ? c->dt_override : c->cfl * c->dx / (O_C * sqrt(2.0));
    s->nsp = c->mode == 0 ? 2 : 1;
    s->w = c->n_atoms * c->dx * c->dx / (double)(c->ppc_ion > 0 ? c->ppc_ion : 1);   /* atoms per metre of y */
    s->r0 = c->r0 > 0 ? c->r0 : pow(c->n_atoms, -1.0 / 3.0);
    s->D = c->D_eV * O_QE;
    /* node sum (units 2^-32 of one macro-atom) -> density in units of n0 = r0^-3 */
    s->rho_scale = s->w / (4294967296.0 * c->dx * c->dx) * pow(s->r0, 3.0);
    s->q[0] = c->ion_charge * O_QE;
    s->m[0] = c->ion_mass_amu * O_AMU;
    s->uth[0] = sqrt(O_KB * c->T_ion_K / (s->m[0] * O_C * O_C));
    s->pair[0] = 1;
    s->q[1] = -O_QE;
    s->m[1] = O_ME;
    s->uth[1] = sqrt(c->T_electron_eV * O_QE / (O_ME * O_C * O_C));
    s->pair[1] = 0;
    size_t nn = (size_t)c->nx * (c->nz + 1);
    for (int f = 0; f < 6; f++) s->F[f] = calloc(nn, sizeof(double));
    for (int f = 0; f < 3; f++) s->J[f] = calloc(nn, sizeof(int64_t));
    s->rho = calloc(nn, sizeof(int64_t));
    /* laser: E0 from the peak intensity, pulse peak at the slab surface at t_peak */
    s->E0 = sqrt(2.0 * c->I0 / (O_EPS0 * O_C));
    s->omega = c->lambda > 0 ? 2.0 * O_PI * O_C / c->lambda : 0.0;
    s->kwave = s->omega / O_C;
    s->jy_bits = oracle_jy_bits((int64_t)c->ppc_ion + (int64_t)c->ppc_electron);
    s->k_ant = c->nz - 2;
    double L = (double)(s->k_ant - c->slab_k) * c->dx;                 /* antenna -> focus */
    s->t_ant = c->t_peak - L / O_C;
    if (c->laser_profile == 2) {
        double zR = O_PI * c->w0 * c->w0 / c->lambda, sa = -L;
        s->w_ant = c->w0 * sqrt(1.0 + (sa / zR) * (sa / zR));
        s->R_ant = sa + zR * zR / sa;
        s->gouy_ant = 0.5 * atan(sa / zR);
        s->amp_ant = sqrt(c->w0 / s->w_ant);
    }
    if (with_particles) init_particles(s);
    else for (int sp = 0; sp < s->nsp; sp++) alloc_species(s, sp, 0);
    redeposit(s);
    return s;
}

void oracle_free(ostate* s)
{
    if (!s) return;
    for (int sp = 0; sp < 2; sp++) { free(s->x[sp]); free(s->z[sp]); free(s->ux[sp]); free(s->uy[sp]); free(s->uz[sp]); }
    for (int f = 0; f < 6; f++) free(s->F[f]);
    for (int f = 0; f < 3; f++) free(s->J[f]);
    free(s->rho);
    free(s);
}

int64_t oracle_num_particles(const ostate* s, int32_t sp) { return sp < s->nsp ? s->np[sp] : 0; }
double oracle_dt(const ostate* s) { return s->dt; }
double oracle_weight(const ostate* s) { return s->w; }
double oracle_rho_scale(const ostate* s) { return s->rho_scale; }
int64_t oracle_step_count(const ostate* s) { return s->step; }

void oracle_get_particles(const ostate* s, int32_t sp, double* x, double* z, double* ux, double* uy, double* uz)
{
    int64_t n = s->np[sp];
    memcpy(x, s->x[sp], sizeof(double) * n); memcpy(z, s->z[sp], sizeof(double) * n);
    memcpy(ux, s->ux[sp], sizeof(double) * n); memcpy(uy, s->uy[sp], sizeof(double) * n);
    memcpy(uz, s->uz[sp], sizeof(double) * n);
}

void oracle_set_particles(ostate* s, int32_t sp, int64_t n, const double* x, const double* z,
                          const double* ux, const double* uy, const double* uz)
{
    alloc_species(s, sp, n);
    memcpy(s->x[sp], x, sizeof(double) * n); memcpy(s->z[sp], z, sizeof(double) * n);
    memcpy(s->ux[sp], ux, sizeof(double) * n); memcpy(s->uy[sp], uy, sizeof(double) * n);
    memcpy(s->uz[sp], uz, sizeof(double) * n);
    if (sp == 0) redeposit(s);
}

void oracle_get_field(const ostate* s, int32_t f, double* out)
{
    memcpy(out, s->F[f], sizeof(double) * (size_t)s->c.nx * (s->c.nz + 1));
}
void oracle_set_field(ostate* s, int32_t f, const double* in)
{
    memcpy(s->F[f], in, sizeof(double) * (size_t)s->c.nx * (s->c.nz + 1));
}
void oracle_get_rho(const ostate* s, int64_t* out) { memcpy(out, s->rho, sizeof(int64_t) * (size_t)s->c.nx * (s->c.nz + 1)); }
void oracle_set_rho(ostate* s, const int64_t* in) { memcpy(s->rho, in, sizeof(int64_t) * (size_t)s->c.nx * (s->c.nz + 1)); }
void oracle_get_current(const ostate* s, int64_t* out3)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    for (int f = 0; f < 3; f++) memcpy(out3 + f * nn, s->J[f], sizeof(int64_t) * nn);
}
void oracle_set_current(ostate* s, const int64_t* in3)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    for (int f = 0; f < 3; f++) memcpy(s->J[f], in3 + f * nn, sizeof(int64_t) * nn);
}
void oracle_set_step(ostate* s, int64_t step) { s->step = step; }

/* per-atom pair force (N) on every macro-ion at its current position */
void oracle_pair_force(const ostate* s, double* F)
{
    for (int64_t p = 0; p < s->np[0]; p++) pair_force_at(s, s->x[0][p], s->z[0][p], F + 3 * p, NULL);
}

/* density and gradient seen by a point (units n0, n0 per cell), for pinning the gather */
void oracle_gather_density(const ostate* s, double x, double z, double out[3])
{
    gather_density(s, x, z, &out[0], &out[1], &out[2]);
}

/* E and B at a point (x, z) in cells: each Yee component interpolated bilinearly from its own
 * staggered positions (paper, the PIC-cycle paragraph: fields interpolated to the particle) */
static void gather_EB(const ostate* s, double x, double z, double E[3], double B[3])
{
    E[0] = gather_field(s, s->F[0], x, z, 0.5, 0.0);
    E[1] = gather_field(s, s->F[1], x, z, 0.0, 0.0);
    E[2] = gather_field(s, s->F[2], x, z, 0.0, 0.5);
    B[0] = gather_field(s, s->F[3], x, z, 0.0, 0.5);
    B[1] = gather_field(s, s->F[4], x, z, 0.5, 0.5);
    B[2] = gather_field(s, s->F[5], x, z, 0.5, 0.0);
}

/* the fields the push sees at (x, z): out = Ex, Ey, Ez, Bx, By, Bz, for pinning the gather */
void oracle_gather_fields(const ostate* s, double x, double z, double out[6])
{
    gather_EB(s, x, z, out, out + 3);
}

/* advance one particle (position in cells, u = gamma v / c) through gather, pair force, Boris and
 * the move with walls, from the context's fields and node density */
static void push_one(const ostate* s, int sp, double* px, double* pz, double u[3])
{
    double x = *px, z = *pz;
    double E[3] = {0, 0, 0}, B[3] = {0, 0, 0}, Fp[3] = {0, 0, 0};
    if (s->c.mode == 0) gather_EB(s, x, z, E, B);
    if (s->pair[sp]) pair_force_at(s, x, z, Fp, NULL);
    oracle_boris(s->q[sp], s->m[sp], s->dt, E, B, Fp, u);
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double xn = x + u[0] * O_C * s->dt / (g * s->c.dx);
    double zn = z + u[2] * O_C * s->dt / (g * s->c.dx);
    if (xn < 0.0) xn += s->c.nx;
    if (xn >= s->c.nx) xn -= s->c.nx;
    if (zn < 0.0) { zn = -zn; u[2] = -u[2]; }
    if (zn >= s->c.nz) { zn = 2.0 * s->c.nz - zn; u[2] = -u[2]; }
    *px = xn; *pz = zn;
}

static void push_particle(ostate* s, int sp, int64_t p)
{
    double u[3] = {s->ux[sp][p], s->uy[sp][p], s->uz[sp][p]};
    push_one(s, sp, &s->x[sp][p], &s->z[sp][p], u);
    s->ux[sp][p] = u[0]; s->uy[sp][p] = u[1]; s->uz[sp][p] = u[2];
}

/* Lattice temperature per cell (paper: the transport run starts from the lattice temperature the
 * laser stage leaves once electrons and lattice have equilibrated): for the N particles of
 * species sp in cell (i, k), T = m c^2 / (3 k_B) * sum |u - mean u|^2 / (N - 1), u = gamma v / c:
 * the thermal spread about the cell's mean flow (unbiased over the cell's sample). Cells with
 * fewer than two particles get 0.
 * out: nz * nx values, index k * nx + i. */
void oracle_cell_temperature(const ostate* s, int32_t sp, double* out)
{
    const ocfg* c = &s->c;
    size_t ncell = (size_t)c->nx * (size_t)c->nz;
    double* acc = calloc(5 * ncell, sizeof(double));
    for (int64_t p = 0; p < s->np[sp]; p++) {
        int64_t i = (int64_t)floor(s->x[sp][p]), k = (int64_t)floor(s->z[sp][p]);
        if (k >= c->nz) k = c->nz - 1;                 /* a particle on the top wall */
        size_t q = (size_t)k * c->nx + (size_t)imod(i, c->nx);
        double ux = s->ux[sp][p], uy = s->uy[sp][p], uz = s->uz[sp][p];
        acc[q] += 1.0;
        acc[ncell + q] += ux;
        acc[2 * ncell + q] += uy;
        acc[3 * ncell + q] += uz;
        acc[4 * ncell + q] += ux * ux + uy * uy + uz * uz;
    }
    double mc2_3k = s->m[sp] * O_C * O_C / (3.0 * O_KB);
    for (size_t q = 0; q < ncell; q++) {
        double n = acc[q];
        if (n < 2.0) { out[q] = 0.0; continue; }
        double mx = acc[ncell + q] / n, my = acc[2 * ncell + q] / n, mz = acc[3 * ncell + q] / n;
        out[q] = mc2_3k * (acc[4 * ncell + q] - n * (mx * mx + my * my + mz * mz)) / (n - 1.0);
    }
    free(acc);
}

/* Re-temper species sp to a temperature map: momenta drawn at the uniform temperature T_from become
 * the same draws at the temperature of their cell (T: nz * nx values): u -> u sqrt(T_cell / T_from). */
void oracle_set_temperature(ostate* s, int32_t sp, const double* T, double T_from)
{
    const ocfg* c = &s->c;
    for (int64_t p = 0; p < s->np[sp]; p++) {
        int64_t i = (int64_t)floor(s->x[sp][p]), k = (int64_t)floor(s->z[sp][p]);
        if (k >= c->nz) k = c->nz - 1;
        double f = sqrt(T[(size_t)k * c->nx + (size_t)imod(i, c->nx)] / T_from);
        s->ux[sp][p] *= f;
        s->uy[sp][p] *= f;
        s->uz[sp][p] *= f;
    }
}

/* Regridding a cell map between stages on different cells (paper: the laser-interaction run, on
 * much finer cells than the transport run, hands over its lattice temperature). The grids are
 * placed on each other by the slab surface and the laser axis: cell (i, j, k) of a grid (nx, ny,
 * nz, dx, surface) spans x in [(i - nx/2) dx, (i + 1 - nx/2) dx], y likewise (3D) and depth
 * [(k - surface) dx, (k + 1 - surface) dx]. Each destination cell takes the volume-weighted mean of
 * the source cells it overlaps, the part of it outside the source grid counting as fill. Written
 * as that definition: the overlap of every destination cell with every source cell. */
static double overlap1(double a0, double a1, double b0, double b1)
{
    const double lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
    return hi > lo ? hi - lo : 0.0;
}

void oracle_regrid_cells(int32_t dims, const double* src, int32_t snx, int32_t sny, int32_t snz, double sdx,
                         int32_t ssurf, double* dst, int32_t dnx, int32_t dny, int32_t dnz, double ddx, int32_t dsurf,
                         double fill)
{
    if (dims == 2) sny = dny = 1;
    const double vol = dims == 3 ? ddx * ddx * ddx : ddx * ddx;
    for (int32_t k = 0; k < dnz; k++)
        for (int32_t j = 0; j < dny; j++)
            for (int32_t i = 0; i < dnx; i++) {
                const double x0 = (i - 0.5 * dnx) * ddx, y0 = (j - 0.5 * dny) * ddx, z0 = (k - dsurf) * ddx;
                double sum = 0.0, covered = 0.0;
                for (int32_t sk = 0; sk < snz; sk++)
                    for (int32_t sj = 0; sj < sny; sj++)
                        for (int32_t si = 0; si < snx; si++) {
                            const double bx = (si - 0.5 * snx) * sdx, by = (sj - 0.5 * sny) * sdx,
                                         bz = (sk - ssurf) * sdx;
                            double w = overlap1(x0, x0 + ddx, bx, bx + sdx) * overlap1(z0, z0 + ddx, bz, bz + sdx);
                            if (dims == 3) w *= overlap1(y0, y0 + ddx, by, by + sdx);
                            if (w > 0.0) {
                                sum += w * src[((size_t)sk * sny + sj) * snx + si];
                                covered += w;
                            }
                        }
                dst[((size_t)k * dny + j) * dnx + i] = (sum + fill * (vol - covered)) / vol;
            }
}

/* Crater profile (paper: after solidification the crater's width and depth are read off the
 * density map): for every node column i, the material missing from the original slab as a
 * thickness of solid-density material (m): dx * sum over node rows k = 0..slab_k of the density
 * drop (rho0 - rho)(k, i) in units of the solid density. rho NULL: the state's own node sums. */
void oracle_crater_profile(const ostate* s, const int64_t* rho0, const int64_t* rho, double* out)
{
    const ocfg* c = &s->c;
    const int64_t* now = rho ? rho : s->rho;
    int top = c->slab_k < c->nz ? c->slab_k : c->nz;
    /* a node sum counts 2^-32 macro-atoms per cell area: density = sum * w / (2^32 dx^2) */
    double to_solid = s->w / (4294967296.0 * c->dx * c->dx) / c->n_atoms;
    for (int i = 0; i < c->nx; i++) {
        int64_t missing = 0;
        for (int k = 0; k <= top; k++) missing += rho0[NODE(s, i, k)] - now[NODE(s, i, k)];
        out[i] = c->dx * ((double)missing * to_solid);
    }
}

/* Initial state of one particle (slot j of cell (i, k)) and one particle's push from the current
 * fields and node density, for checking sampled particles of large runs one by one.
 * v: x, z, ux, uy, uz (the push updates it in place). */
void oracle_init_particle(const ostate* s, int32_t sp, int64_t i, int64_t k, int64_t j, double* v)
{
    init_one(s, sp, i, k, j, v);
}

void oracle_push_one(const ostate* s, int32_t sp, double* v)
{
    double u[3] = {v[2], v[3], v[4]};
    push_one(s, sp, &v[0], &v[1], u);
    v[2] = u[0]; v[3] = u[1]; v[4] = u[2];
}

/* The Maxwell part of the cycle alone, from the stored current (for checking a field update
 * against a current computed elsewhere). */
void oracle_maxwell(ostate* s)
{
    half_step_B(s);
    full_step_E(s);
    half_step_B(s);
}

/* One PIC cycle (paper, PIC-cycle paragraph): pair force from the node density at x^n,
 * Lorentz + pair push, current from x^n -> x^(n+1), node density at x^(n+1), Maxwell. */
void oracle_step(ostate* s, int32_t nsteps)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    for (int it = 0; it < nsteps; it++) {
        for (int f = 0; f < 3; f++) memset(s->J[f], 0, sizeof(int64_t) * nn);
        for (int sp = 0; sp < s->nsp; sp++) {
            int64_t n = s->np[sp];
            double* x0 = malloc(sizeof(double) * (n ? n : 1));
            double* z0 = malloc(sizeof(double) * (n ? n : 1));
            memcpy(x0, s->x[sp], sizeof(double) * n);
            memcpy(z0, s->z[sp], sizeof(double) * n);
            for (int64_t p = 0; p < n; p++) push_particle(s, sp, p);      /* uses rho at x^n */
            if (s->c.mode == 0 && s->q[sp] != 0.0) {
                int sign = s->q[sp] > 0 ? 1 : -1;
                for (int64_t p = 0; p < n; p++) {
                    float fux = (float)s->ux[sp][p], fuy = (float)s->uy[sp][p], fuz = (float)s->uz[sp][p];
                    oracle_deposit_current(s->c.nx, s->c.nz, 1, sign, x0 + p, z0 + p, s->x[sp] + p, s->z[sp] + p,
                                           &fux, &fuy, &fuz, s->jy_bits, s->J[0], s->J[1], s->J[2]);
                }
            }
            free(x0); free(z0);
        }
        redeposit(s);                                                    /* rho at x^(n+1) */
        if (s->c.mode == 0) {
            half_step_B(s);
            full_step_E(s);
            half_step_B(s);
        }
        s->step++;
    }
}

/* Energies (J per metre of y): out = {kinetic ions, kinetic electrons, field E, field B, pair}.
 * Kinetic uses the stored u (half step); field energy weights the wall node rows by 1/2. */
void oracle_energy(const ostate* s, double out[5])
{
    for (int i = 0; i < 5; i++) out[i] = 0.0;
    for (int sp = 0; sp < s->nsp; sp++) {
        double acc = 0.0;
        for (int64_t p = 0; p < s->np[sp]; p++) {
            double u2 = s->ux[sp][p] * s->ux[sp][p] + s->uy[sp][p] * s->uy[sp][p] + s->uz[sp][p] * s->uz[sp][p];
            acc += u2 / (sqrt(1.0 + u2) + 1.0);
        }
        out[sp] = acc * s->w * s->m[sp] * O_C * O_C;
    }
    int nx = s->c.nx, nz = s->c.nz;
    double vol = s->c.dx * s->c.dx, mu0 = 1.0 / (O_EPS0 * O_C * O_C);
    double eE = 0.0, eB = 0.0;
    for (int k = 0; k <= nz; k++) {
        double wn = (k == 0 || k == nz) ? 0.5 : 1.0;       /* node-row components */
        for (int i = 0; i < nx; i++) {
            size_t c = NODE(s, i, k);
            eE += wn * (s->F[0][c] * s->F[0][c] + s->F[1][c] * s->F[1][c]);
            eB += wn * s->F[5][c] * s->F[5][c];
            if (k < nz) {
                eE += s->F[2][c] * s->F[2][c];
                eB += s->F[3][c] * s->F[3][c] + s->F[4][c] * s->F[4][c];
            }
        }
    }
    out[2] = 0.5 * O_EPS0 * eE * vol;
    out[3] = 0.5 / mu0 * eB * vol;
    double pe = 0.0;
    for (int64_t p = 0; p < s->np[0]; p++) {
        double F[3], e;
        pair_force_at(s, s->x[0][p], s->z[0][p], F, &e);
        pe += e;
    }
    out[4] = pe * s->w;
}

/* E_x the antenna launches at (x in cells, t), for pinning the source */
double oracle_laser_field(const ostate* s, double x_cells, double t) { return laser_field(s, x_cells, t); }

/* ======================================================================================== */
/* 3D3V cycle (the paper's method in three dimensions: Eqs. (1)-(3) along x, y and z, the    */
/* cubic lattice's six neighbours). Fixed point 2^14 per axis keeps the int64 sums far from  */
/* overflow (a particle's weight product is at most 2^42).                                   */
/* Grids: (nz+1) node rows of ny x nx, index (k*ny + j)*nx + i. Yee positions: Ex (i+1/2,j,k) */
/* Ey (i,j+1/2,k) Ez (i,j,k+1/2) Bx (i,j+1/2,k+1/2) By (i+1/2,j,k+1/2) Bz (i+1/2,j+1/2,k).   */
/* x and y periodic, walls at z = 0 and z = nz.                                               */
/* ======================================================================================== */
#define Q3 16384LL

typedef struct {
    int32_t nx, ny, nz, slab_k, mode, ppc_ion, ppc_electron, pot_mode, laser_profile;
    double dx, cfl, dt_override, n_atoms, T_ion_K, T_electron_eV, ion_charge, ion_mass_amu;
    double D_eV, r0, c_att, s_rep, lambda, I0, tau_fwhm, w0, t_peak;
    uint64_t seed;
    int32_t temp_profile;    /* 0: uniform T_ion_K; 1: lattice temperature of a laser spot       */
    int32_t lattice;
    double T_spot_K, spot_w, spot_depth;
    double morse_a;
    double eam_ec, eam_phi, eam_alpha, eam_beta, eam_gamma;
} ocfg3;

typedef struct {
    ocfg3 c;
    double dt, w, r0, D, rho_scale;
    int nsp;
    double q[2], m[2], uth[2];
    int64_t np[2];
    double *x[2], *y[2], *z[2], *ux[2], *uy[2], *uz[2];
    double *F[6];
    int64_t *rho, *J[3];
    int64_t step;
    double E0, omega, kwave, t_ant, w_ant, R_ant, gouy_ant, amp_ant;
    int k_ant;
    double injected;                    /* energy through the plane below the antenna (J)   */
} ostate3;

static int64_t hat3q(int64_t X, int64_t j) { int64_t d = X - Q3 * j; if (d < 0) d = -d; return d < Q3 ? Q3 - d : 0; }
#define N3(s, i, j, k) (((size_t)(k) * (size_t)(s)->c.ny + (size_t)(j)) * (size_t)(s)->c.nx + (size_t)(i))
static size_t nn3(const ostate3* s) { return (size_t)s->c.nx * s->c.ny * (s->c.nz + 1); }

/* node density: weights to the 8 nearest nodes */
void oracle3_deposit_density(int32_t nx, int32_t ny, int32_t nz, int64_t n, const double* x, const double* y,
                             const double* z, int64_t* rho)
{
    memset(rho, 0, sizeof(int64_t) * (size_t)nx * ny * (nz + 1));
    for (int64_t p = 0; p < n; p++) {
        int64_t X = llrint(x[p] * (double)Q3), Y = llrint(y[p] * (double)Q3), Z = llrint(z[p] * (double)Q3);
        int64_t i0 = floordiv(X, Q3), j0 = floordiv(Y, Q3), l0 = floordiv(Z, Q3);
        for (int64_t l = l0; l <= l0 + 1; l++)
            for (int64_t j = j0; j <= j0 + 1; j++)
                for (int64_t i = i0; i <= i0 + 1; i++) {
                    int64_t w = hat3q(X, i) * hat3q(Y, j) * hat3q(Z, l);
                    if (w == 0) continue;
                    if (l < 0 || l > nz) abort();
                    rho[((size_t)l * ny + imod(j, ny)) * nx + imod(i, nx)] += w;
                }
    }
}

/* Esirkepov current in 3D for linear weights:
 *   6 Wx = dSx (2 S0y S0z + S1y S0z + S0y S1z + 2 S1y S1z)   (and cyclically)
 *   J6x(i+1/2) = J6x(i-1/2) - 6 Wx(i)  along each x line
 * so that 6 (rho1 - rho0) + div(J6) = 0 in integers (units 2^-42). */
static void deposit_current3_one(int nx, int ny, int nz, int64_t* J6x, int64_t* J6y, int64_t* J6z, int64_t sign,
                                 int64_t X0, int64_t Y0, int64_t Z0, int64_t X1, int64_t Y1, int64_t Z1)
{
    int64_t bx = floordiv(X0 < X1 ? X0 : X1, Q3), by = floordiv(Y0 < Y1 ? Y0 : Y1, Q3), bz = floordiv(Z0 < Z1 ? Z0 : Z1, Q3);
    int64_t S0x[3], S1x[3], S0y[3], S1y[3], S0z[3], S1z[3];
    for (int a = 0; a < 3; a++) {
        S0x[a] = hat3q(X0, bx + a); S1x[a] = hat3q(X1, bx + a);
        S0y[a] = hat3q(Y0, by + a); S1y[a] = hat3q(Y1, by + a);
        S0z[a] = hat3q(Z0, bz + a); S1z[a] = hat3q(Z1, bz + a);
    }
    for (int c = 0; c < 3; c++)                /* J_x along x lines (b = y, c = z) */
        for (int b = 0; b < 3; b++) {
            int64_t P = 2 * S0y[b] * S0z[c] + S1y[b] * S0z[c] + S0y[b] * S1z[c] + 2 * S1y[b] * S1z[c];
            int64_t acc = 0;
            for (int a = 0; a < 2; a++) {
                acc -= (S1x[a] - S0x[a]) * P;
                if (acc != 0) {
                    int64_t l = bz + c;
                    if (l < 0 || l > nz) abort();
                    J6x[((size_t)l * ny + imod(by + b, ny)) * nx + imod(bx + a, nx)] += sign * acc;
                }
            }
        }
    for (int c = 0; c < 3; c++)                /* J_y along y lines */
        for (int a = 0; a < 3; a++) {
            int64_t P = 2 * S0x[a] * S0z[c] + S1x[a] * S0z[c] + S0x[a] * S1z[c] + 2 * S1x[a] * S1z[c];
            int64_t acc = 0;
            for (int b = 0; b < 2; b++) {
                acc -= (S1y[b] - S0y[b]) * P;
                if (acc != 0) {
                    int64_t l = bz + c;
                    if (l < 0 || l > nz) abort();
                    J6y[((size_t)l * ny + imod(by + b, ny)) * nx + imod(bx + a, nx)] += sign * acc;
                }
            }
        }
    for (int b = 0; b < 3; b++)                /* J_z along z lines */
        for (int a = 0; a < 3; a++) {
            int64_t P = 2 * S0x[a] * S0y[b] + S1x[a] * S0y[b] + S0x[a] * S1y[b] + 2 * S1x[a] * S1y[b];
            int64_t acc = 0;
            for (int c = 0; c < 2; c++) {
                acc -= (S1z[c] - S0z[c]) * P;
                if (acc != 0) {
                    int64_t l = bz + c;
                    if (l < 0 || l > nz - 1) abort();
                    J6z[((size_t)l * ny + imod(by + b, ny)) * nx + imod(bx + a, nx)] += sign * acc;
                }
            }
        }
}

void oracle3_deposit_current(int32_t nx, int32_t ny, int32_t nz, int64_t n, int32_t sign, const double* x0,
                             const double* y0, const double* z0, const double* x1, const double* y1, const double* z1,
                             int64_t* J6x, int64_t* J6y, int64_t* J6z)
{
    int64_t Px = (int64_t)nx * Q3, Py = (int64_t)ny * Q3;
    for (int64_t p = 0; p < n; p++) {
        int64_t X0 = llrint(x0[p] * (double)Q3), Y0 = llrint(y0[p] * (double)Q3), Z0 = llrint(z0[p] * (double)Q3);
        int64_t X1 = llrint(x1[p] * (double)Q3), Y1 = llrint(y1[p] * (double)Q3), Z1 = llrint(z1[p] * (double)Q3);
        while (X1 - X0 > Px / 2) X1 -= Px;
        while (X0 - X1 > Px / 2) X1 += Px;
        while (Y1 - Y0 > Py / 2) Y1 -= Py;
        while (Y0 - Y1 > Py / 2) Y1 += Py;
        deposit_current3_one(nx, ny, nz, J6x, J6y, J6z, sign, X0, Y0, Z0, X1, Y1, Z1);
    }
}

static double nhat3(const ostate3* s, int64_t i, int64_t j, int64_t k)
{
    double v = (double)s->rho[N3(s, imod(i, s->c.nx), imod(j, s->c.ny), k)] * s->rho_scale;
    if (k == 0 || k == s->c.nz) v *= 2.0;
    return v;
}

/* trilinear density and its exact gradient (per cell) */
static void gather_density3(const ostate3* s, double x, double y, double z, double* n, double g[3])
{
    int64_t i = (int64_t)floor(x), j = (int64_t)floor(y), k = (int64_t)floor(z);
    double f[3] = {x - (double)i, y - (double)j, z - (double)k};
    if (k >= s->c.nz) { k = s->c.nz - 1; f[2] = 1.0; }
    double v[2][2][2];
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) v[c][b][a] = nhat3(s, i + a, j + b, k + c);
    *n = 0.0; g[0] = g[1] = g[2] = 0.0;
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) {
                double wx = a ? f[0] : 1 - f[0], wy = b ? f[1] : 1 - f[1], wz = c ? f[2] : 1 - f[2];
                double sx = a ? 1.0 : -1.0, sy = b ? 1.0 : -1.0, sz = c ? 1.0 : -1.0;
                *n += wx * wy * wz * v[c][b][a];
                g[0] += sx * wy * wz * v[c][b][a];
                g[1] += wx * sy * wz * v[c][b][a];
                g[2] += wx * wy * sz * v[c][b][a];
            }
}

static double gather_field3(const ostate3* s, const double* A, double x, double y, double z, double sx, double sy, double sz)
{
    int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    double xs = x - sx, ys = y - sy, zs = z - sz;
    int64_t rows = sz > 0 ? nz : nz + 1;
    if (zs < 0.0) zs = 0.0;
    if (zs > (double)(rows - 1)) zs = (double)(rows - 1);
    int64_t i = (int64_t)floor(xs), j = (int64_t)floor(ys), k = (int64_t)floor(zs);
    double fx = xs - i, fy = ys - j, fz = zs - k;
    if (k >= rows - 1) { k = rows - 2; fz = 1.0; }
    double v = 0.0;
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) {
                double w = (a ? fx : 1 - fx) * (b ? fy : 1 - fy) * (c ? fz : 1 - fz);
                v += w * A[((size_t)(k + c) * ny + imod(j + b, ny)) * nx + imod(i + a, nx)];
            }
    return v;
}

/* Eqs. (1)-(3) along x, y and z; energy = half the sum of U over the six neighbours */
static void pair_force3_at(const ostate3* s, double x, double y, double z, double F[3], double* energy)
{
    double n, g[3];
    gather_density3(s, x, y, z, &n, g);
    F[0] = F[1] = F[2] = 0.0;
    if (energy) *energy = 0.0;
    if (!(n > 0.0)) return;
    double r0_dx = s->r0 / s->c.dx, f_unit = s->D / s->r0, u = 0.0;
    int pm = s->c.pot_mode;
    if (pm == 3) {
        eam_p p = eam_params(s->c.D_eV, s->c.eam_ec, s->c.eam_phi, s->c.eam_alpha, s->c.eam_beta, s->c.eam_gamma);
        double Fu[3];
        eam_atom(&p, n, g, 1, r0_dx, Fu, &u);
        for (int d = 0; d < 3; d++) F[d] = f_unit * Fu[d];
        if (energy) *energy = s->D * u;
        return;
    }
    if (s->c.lattice == 1) {
        double Fu[3];
        lattice_pair(1, pm, s->c.c_att, s->c.s_rep, s->c.morse_a, n, g, r0_dx, Fu, &u);
        for (int d = 0; d < 3; d++) F[d] = f_unit * Fu[d];
        if (energy) *energy = s->D * u;
        return;
    }
    for (int d = 0; d < 3; d++) {
        double ap, am;
        oracle_neighbor_distances(n, g[d], r0_dx, &ap, &am);
        double dUp = isinf(ap) ? 0.0 : pot_dU(pm, s->c.c_att, s->c.s_rep, s->c.morse_a, ap);
        double dUm = isinf(am) ? 0.0 : pot_dU(pm, s->c.c_att, s->c.s_rep, s->c.morse_a, am);
        F[d] = f_unit * (dUp - dUm);
        if (!isinf(ap)) u += pot_U(pm, s->c.c_att, s->c.s_rep, s->c.morse_a, ap);
        if (!isinf(am)) u += pot_U(pm, s->c.c_att, s->c.s_rep, s->c.morse_a, am);
    }
    if (energy) *energy = 0.5 * s->D * u;
}

static double laser_field3(const ostate3* s, double x_cells, double y_cells, double t)
{
    if (s->c.laser_profile == 0) return 0.0;
    double tau = t - s->t_ant;
    double env = exp(-2.0 * log(2.0) * tau * tau / (s->c.tau_fwhm * s->c.tau_fwhm));
    if (s->c.laser_profile == 1) return s->E0 * env * sin(s->omega * tau);
    double xr = (x_cells - 0.5 * s->c.nx) * s->c.dx, yr = (y_cells - 0.5 * s->c.ny) * s->c.dx;
    double r2 = xr * xr + yr * yr;
    double amp = s->amp_ant * exp(-r2 / (s->w_ant * s->w_ant));
    double phase = -s->kwave * r2 / (2.0 * s->R_ant) + s->gouy_ant;
    return s->E0 * amp * env * sin(s->omega * tau + phase);
}

/* 3D Yee: B half step, E step, B half step */
static void half_step_B3(ostate3* s)
{
    int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    double h = 0.5 * s->dt / s->c.dx;
    double *Ex = s->F[0], *Ey = s->F[1], *Ez = s->F[2], *Bx = s->F[3], *By = s->F[4], *Bz = s->F[5];
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int ip = (i + 1) % nx, jp = (j + 1) % ny;
                size_t c = N3(s, i, j, k);
                if (k < nz) {
                    /* dBx/dt = dEy/dz - dEz/dy ; dBy/dt = dEz/dx - dEx/dz */
                    Bx[c] += h * ((Ey[N3(s, i, j, k + 1)] - Ey[c]) - (Ez[N3(s, i, jp, k)] - Ez[c]));
                    By[c] += h * ((Ez[N3(s, ip, j, k)] - Ez[c]) - (Ex[N3(s, i, j, k + 1)] - Ex[c]));
                }
                /* dBz/dt = dEx/dy - dEy/dx */
                Bz[c] += h * ((Ex[N3(s, i, jp, k)] - Ex[c]) - (Ey[N3(s, ip, j, k)] - Ey[c]));
            }
}

static void full_step_E3(ostate3* s)
{
    int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    double cdt = O_C * s->dt, h = O_C * O_C * s->dt / s->c.dx;
    double *Ex = s->F[0], *Ey = s->F[1], *Ez = s->F[2], *Bx = s->F[3], *By = s->F[4], *Bz = s->F[5];
    size_t nn = nn3(s);
    double* nEx = malloc(sizeof(double) * nn);
    double* nEy = malloc(sizeof(double) * nn);
    double cj = O_QE * s->w / (6.0 * 4398046511104.0 * s->c.dx * s->c.dx * O_EPS0);    /* 6 * 2^42 */
    double tmid = ((double)s->step + 0.5) * s->dt;
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int im = (i + nx - 1) % nx, jm = (j + ny - 1) % ny;
                size_t c = N3(s, i, j, k);
                nEx[c] = Ex[c];
                nEy[c] = Ey[c];
                if (k > 0 && k < nz) {
                    /* dEx/dt = c^2 (dBz/dy - dBy/dz) - Jx/eps0 ; dEy/dt = c^2 (dBx/dz - dBz/dx) - Jy/eps0 */
                    nEx[c] = Ex[c] + h * ((Bz[c] - Bz[N3(s, i, jm, k)]) - (By[c] - By[N3(s, i, j, k - 1)])) - cj * (double)s->J[0][c];
                    nEy[c] = Ey[c] + h * ((Bx[c] - Bx[N3(s, i, j, k - 1)]) - (Bz[c] - Bz[N3(s, im, j, k)])) - cj * (double)s->J[1][c];
                    if (k == s->k_ant) nEx[c] += 2.0 * (cdt / s->c.dx) * laser_field3(s, (double)i + 0.5, (double)j, tmid);
                }
            }
    double alpha = (cdt - s->c.dx) / (cdt + s->c.dx);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t b0 = N3(s, i, j, 0), b1 = N3(s, i, j, 1), t0 = N3(s, i, j, nz), t1 = N3(s, i, j, nz - 1);
            nEx[b0] = Ex[b1] + alpha * (nEx[b1] - Ex[b0]);
            nEy[b0] = Ey[b1] + alpha * (nEy[b1] - Ey[b0]);
            nEx[t0] = Ex[t1] + alpha * (nEx[t1] - Ex[t0]);
            nEy[t0] = Ey[t1] + alpha * (nEy[t1] - Ey[t0]);
        }
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int im = (i + nx - 1) % nx, jm = (j + ny - 1) % ny;
                size_t c = N3(s, i, j, k);
                /* dEz/dt = c^2 (dBy/dx - dBx/dy) - Jz/eps0 */
                Ez[c] += h * ((By[c] - By[N3(s, im, j, k)]) - (Bx[c] - Bx[N3(s, i, jm, k)])) - cj * (double)s->J[2][c];
            }
    /* injected energy through the node plane below the antenna (as in 2D, per cell area dx^2) */
    int kp = s->k_ant - 1;
    if (kp >= 1 && kp < nz) {
        double mu0 = 1.0 / (O_EPS0 * O_C * O_C), sum = 0.0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = N3(s, i, j, kp), d = N3(s, i, j, kp - 1);
                double ex = 0.5 * (Ex[c] + nEx[c]), ey = 0.5 * (Ey[c] + nEy[c]);
                sum += ex * 0.5 * (By[d] + By[c]) - ey * 0.5 * (Bx[d] + Bx[c]);
            }
        s->injected -= sum / mu0 * s->c.dx * s->c.dx * s->dt;
    }
    memcpy(Ex, nEx, sizeof(double) * nn);
    memcpy(Ey, nEy, sizeof(double) * nn);
    free(nEx); free(nEy);
}

double oracle3_injected(const ostate3* s) { return s->injected; }

static void alloc_species3(ostate3* s, int sp, int64_t n)
{
    free(s->x[sp]); free(s->y[sp]); free(s->z[sp]); free(s->ux[sp]); free(s->uy[sp]); free(s->uz[sp]);
    s->np[sp] = n;
    size_t b = sizeof(double) * (size_t)(n > 0 ? n : 1);
    s->x[sp] = calloc(1, b); s->y[sp] = calloc(1, b); s->z[sp] = calloc(1, b);
    s->ux[sp] = calloc(1, b); s->uy[sp] = calloc(1, b); s->uz[sp] = calloc(1, b);
}

static void redeposit3(ostate3* s)
{
    oracle3_deposit_density(s->c.nx, s->c.ny, s->c.nz, s->np[0], s->x[0], s->y[0], s->z[0], s->rho);
}

/* initial slab: cell rows k < slab_k over all (i, j); positions draws 0 (x), 6 (y), 1 (z) */
/* initial state of the particle in slot q of cell (i, j, k): x, y, z, ux, uy, uz */
/* The laser-spot lattice temperature of the 2D start (Fig. 2 and the initialisation of the
   atomic-transport run) around an axis through the middle of the x-y plane: the Gaussian's
   argument is the squared radius from the axis. */
static double spot_temperature3(const ocfg3* c, double x, double y, double z)
{
    double rx = (x - 0.5 * c->nx) * c->dx / c->spot_w;
    double ry = (y - 0.5 * c->ny) * c->dx / c->spot_w;
    double depth = (c->slab_k - z) * c->dx / c->spot_depth;
    return c->T_ion_K + (c->T_spot_K - c->T_ion_K) * exp(-2.0 * (rx * rx + ry * ry)) * exp(-depth);
}

static void init_one3(const ostate3* s, int sp, int64_t i, int64_t j, int64_t k, int64_t q, double out[6])
{
    const ocfg3* c = &s->c;
    int ppc = sp == 0 ? c->ppc_ion : c->ppc_electron;
    uint64_t cellidx = ((uint64_t)k * c->ny + (uint64_t)j) * (uint64_t)c->nx + (uint64_t)i;
    int pos_sp = (sp == 1 && c->ppc_electron == c->ppc_ion) ? 0 : sp;
    uint64_t pid = cellidx * (uint64_t)ppc + (uint64_t)q;
    out[0] = (double)i + draw_unit24(draw_bits(c->seed, pos_sp, pid, 0));
    out[1] = (double)j + draw_unit24(draw_bits(c->seed, pos_sp, pid, 6));
    out[2] = (double)k + draw_unit24(draw_bits(c->seed, pos_sp, pid, 1));
    double r1 = sqrt(-2.0 * log(draw_open53(draw_bits(c->seed, sp, pid, 2))));
    double a1 = 2.0 * O_PI * draw_unit24(draw_bits(c->seed, sp, pid, 3));
    double r2 = sqrt(-2.0 * log(draw_open53(draw_bits(c->seed, sp, pid, 4))));
    double a2 = 2.0 * O_PI * draw_unit24(draw_bits(c->seed, sp, pid, 5));
    double uth = s->uth[sp];
    if (sp == 0 && c->temp_profile == 1)
        uth = sqrt(O_KB * spot_temperature3(c, out[0], out[1], out[2]) / (s->m[0] * O_C * O_C));
    out[3] = uth * r1 * cos(a1);
    out[4] = uth * r1 * sin(a1);
    out[5] = uth * r2 * cos(a2);
}

static void init_particles3(ostate3* s)
{
    const ocfg3* c = &s->c;
    int64_t ncell = (int64_t)c->nx * c->ny * c->slab_k;
    for (int sp = 0; sp < s->nsp; sp++) {
        int ppc = sp == 0 ? c->ppc_ion : c->ppc_electron;
        alloc_species3(s, sp, ncell * ppc);
        int64_t p = 0;
        for (int k = 0; k < c->slab_k; k++)
            for (int j = 0; j < c->ny; j++)
                for (int i = 0; i < c->nx; i++)
                    for (int q = 0; q < ppc; q++, p++) {
                        double v[6];
                        init_one3(s, sp, i, j, k, q, v);
                        s->x[sp][p] = v[0]; s->y[sp][p] = v[1]; s->z[sp][p] = v[2];
                        s->ux[sp][p] = v[3]; s->uy[sp][p] = v[4]; s->uz[sp][p] = v[5];
                    }
    }
}

ostate3* oracle3_create(const ocfg3* cfg, int32_t with_particles)
{
    ostate3* s = calloc(1, sizeof(ostate3));
    s->c = *cfg;
    const ocfg3* c = &s->c;
    s->dt = c->dt_override > 0 ? c->dt_override : c->cfl * c->dx / (O_C * sqrt(3.0));
    s->nsp = c->mode == 0 ? 2 : 1;
    s->w = c->n_atoms * c->dx * c->dx * c->dx / (double)(c->ppc_ion > 0 ? c->ppc_ion : 1);
    s->r0 = c->r0 > 0 ? c->r0 : pow(c->n_atoms, -1.0 / 3.0);
    s->D = c->D_eV * O_QE;
    s->rho_scale = s->w / (4398046511104.0 * c->dx * c->dx * c->dx) * pow(s->r0, 3.0);   /* 2^42 */
    s->q[0] = c->ion_charge * O_QE; s->m[0] = c->ion_mass_amu * O_AMU;
    s->uth[0] = sqrt(O_KB * c->T_ion_K / (s->m[0] * O_C * O_C));
    s->q[1] = -O_QE; s->m[1] = O_ME;
    s->uth[1] = sqrt(c->T_electron_eV * O_QE / (O_ME * O_C * O_C));
    size_t nn = nn3(s);
    for (int f = 0; f < 6; f++) s->F[f] = calloc(nn, sizeof(double));
    for (int f = 0; f < 3; f++) s->J[f] = calloc(nn, sizeof(int64_t));
    s->rho = calloc(nn, sizeof(int64_t));
    s->E0 = sqrt(2.0 * c->I0 / (O_EPS0 * O_C));
    s->omega = c->lambda > 0 ? 2.0 * O_PI * O_C / c->lambda : 0.0;
    s->kwave = s->omega / O_C;
    s->k_ant = c->nz - 2;
    double L = (double)(s->k_ant - c->slab_k) * c->dx;
    s->t_ant = c->t_peak - L / O_C;
    if (c->laser_profile == 2) {
        /* 3D paraxial Gaussian beam converging on the slab surface */
        double zR = O_PI * c->w0 * c->w0 / c->lambda, sa = -L;
        s->w_ant = c->w0 * sqrt(1.0 + (sa / zR) * (sa / zR));
        s->R_ant = sa + zR * zR / sa;
        s->gouy_ant = atan(sa / zR);
        s->amp_ant = c->w0 / s->w_ant;
    }
    if (with_particles) init_particles3(s);
    else for (int sp = 0; sp < s->nsp; sp++) alloc_species3(s, sp, 0);
    redeposit3(s);
    return s;
}

void oracle3_free(ostate3* s)
{
    if (!s) return;
    for (int sp = 0; sp < 2; sp++) { free(s->x[sp]); free(s->y[sp]); free(s->z[sp]); free(s->ux[sp]); free(s->uy[sp]); free(s->uz[sp]); }
    for (int f = 0; f < 6; f++) free(s->F[f]);
    for (int f = 0; f < 3; f++) free(s->J[f]);
    free(s->rho);
    free(s);
}

int64_t oracle3_num_particles(const ostate3* s, int32_t sp) { return sp < s->nsp ? s->np[sp] : 0; }
double oracle3_dt(const ostate3* s) { return s->dt; }
double oracle3_weight(const ostate3* s) { return s->w; }
double oracle3_rho_scale(const ostate3* s) { return s->rho_scale; }

/* Crater profile in 3D (the density-map measurement of the crater, Eq. 5's diameter): material
 * missing from node column (i, j) of the original slab rows 0..slab_k between the node sums rho0
 * and rho (NULL: the state's own), in metres of solid-density material; out is (ny, nx). A node
 * sum counts 2^-42 macro-atoms per cell volume. */
void oracle3_crater_profile(const ostate3* s, const int64_t* rho0, const int64_t* rho, double* out)
{
    const ocfg3* c = &s->c;
    const int64_t* now = rho ? rho : s->rho;
    int top = c->slab_k < c->nz ? c->slab_k : c->nz;
    double to_solid = s->w / (4398046511104.0 * c->dx * c->dx * c->dx) / c->n_atoms;
    for (int j = 0; j < c->ny; j++)
        for (int i = 0; i < c->nx; i++) {
            int64_t missing = 0;
            for (int k = 0; k <= top; k++) missing += rho0[N3(s, i, j, k)] - now[N3(s, i, j, k)];
            out[(size_t)j * c->nx + i] = c->dx * ((double)missing * to_solid);
        }
}

void oracle3_set_step(ostate3* s, int64_t step) { s->step = step; }

void oracle3_get_particles(const ostate3* s, int32_t sp, double* x, double* y, double* z, double* ux, double* uy, double* uz)
{
    size_t b = sizeof(double) * (size_t)s->np[sp];
    memcpy(x, s->x[sp], b); memcpy(y, s->y[sp], b); memcpy(z, s->z[sp], b);
    memcpy(ux, s->ux[sp], b); memcpy(uy, s->uy[sp], b); memcpy(uz, s->uz[sp], b);
}

void oracle3_set_particles(ostate3* s, int32_t sp, int64_t n, const double* x, const double* y, const double* z,
                           const double* ux, const double* uy, const double* uz)
{
    alloc_species3(s, sp, n);
    size_t b = sizeof(double) * (size_t)n;
    memcpy(s->x[sp], x, b); memcpy(s->y[sp], y, b); memcpy(s->z[sp], z, b);
    memcpy(s->ux[sp], ux, b); memcpy(s->uy[sp], uy, b); memcpy(s->uz[sp], uz, b);
    if (sp == 0) redeposit3(s);
}

void oracle3_get_field(const ostate3* s, int32_t f, double* out) { memcpy(out, s->F[f], sizeof(double) * nn3(s)); }
void oracle3_set_field(ostate3* s, int32_t f, const double* in) { memcpy(s->F[f], in, sizeof(double) * nn3(s)); }
void oracle3_get_rho(const ostate3* s, int64_t* out) { memcpy(out, s->rho, sizeof(int64_t) * nn3(s)); }
void oracle3_set_rho(ostate3* s, const int64_t* in) { memcpy(s->rho, in, sizeof(int64_t) * nn3(s)); }
void oracle3_get_current(const ostate3* s, int64_t* out3)
{
    for (int f = 0; f < 3; f++) memcpy(out3 + f * nn3(s), s->J[f], sizeof(int64_t) * nn3(s));
}
void oracle3_set_current(ostate3* s, const int64_t* in3)
{
    for (int f = 0; f < 3; f++) memcpy(s->J[f], in3 + f * nn3(s), sizeof(int64_t) * nn3(s));
}

void oracle3_pair_force(const ostate3* s, double* F)
{
    for (int64_t p = 0; p < s->np[0]; p++) pair_force3_at(s, s->x[0][p], s->y[0][p], s->z[0][p], F + 3 * p, NULL);
}

void oracle3_maxwell(ostate3* s)
{
    half_step_B3(s);
    full_step_E3(s);
    half_step_B3(s);
}

/* 3D E and B at (x, y, z): trilinear interpolation of each component from its own staggered
 * positions */
static void gather_EB3(const ostate3* s, double x, double y, double z, double E[3], double B[3])
{
    E[0] = gather_field3(s, s->F[0], x, y, z, 0.5, 0.0, 0.0);
    E[1] = gather_field3(s, s->F[1], x, y, z, 0.0, 0.5, 0.0);
    E[2] = gather_field3(s, s->F[2], x, y, z, 0.0, 0.0, 0.5);
    B[0] = gather_field3(s, s->F[3], x, y, z, 0.0, 0.5, 0.5);
    B[1] = gather_field3(s, s->F[4], x, y, z, 0.5, 0.0, 0.5);
    B[2] = gather_field3(s, s->F[5], x, y, z, 0.5, 0.5, 0.0);
}

void oracle3_gather_fields(const ostate3* s, double x, double y, double z, double out[6])
{
    gather_EB3(s, x, y, z, out, out + 3);
}

static void push_one3(const ostate3* s, int sp, double* px, double* py, double* pz, double u[3])
{
    double x = *px, y = *py, z = *pz;
    double E[3] = {0, 0, 0}, B[3] = {0, 0, 0}, Fp[3] = {0, 0, 0};
    if (s->c.mode == 0) gather_EB3(s, x, y, z, E, B);
    if (sp == 0) pair_force3_at(s, x, y, z, Fp, NULL);
    oracle_boris(s->q[sp], s->m[sp], s->dt, E, B, Fp, u);
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double k = O_C * s->dt / (g * s->c.dx);
    double xn = x + u[0] * k, yn = y + u[1] * k, zn = z + u[2] * k;
    if (xn < 0.0) xn += s->c.nx;
    if (xn >= s->c.nx) xn -= s->c.nx;
    if (yn < 0.0) yn += s->c.ny;
    if (yn >= s->c.ny) yn -= s->c.ny;
    if (zn < 0.0) { zn = -zn; u[2] = -u[2]; }
    if (zn >= s->c.nz) { zn = 2.0 * s->c.nz - zn; u[2] = -u[2]; }
    *px = xn; *py = yn; *pz = zn;
}

static void push_particle3(ostate3* s, int sp, int64_t p)
{
    double u[3] = {s->ux[sp][p], s->uy[sp][p], s->uz[sp][p]};
    push_one3(s, sp, &s->x[sp][p], &s->y[sp][p], &s->z[sp][p], u);
    s->ux[sp][p] = u[0]; s->uy[sp][p] = u[1]; s->uz[sp][p] = u[2];
}

/* one particle's initial state and push in 3D; v: x, y, z, ux, uy, uz */
void oracle3_init_particle(const ostate3* s, int32_t sp, int64_t i, int64_t j, int64_t k, int64_t q, double* v)
{
    init_one3(s, sp, i, j, k, q, v);
}

void oracle3_push_one(const ostate3* s, int32_t sp, double* v)
{
    double u[3] = {v[3], v[4], v[5]};
    push_one3(s, sp, &v[0], &v[1], &v[2], u);
    v[3] = u[0]; v[4] = u[1]; v[5] = u[2];
}

void oracle3_step(ostate3* s, int32_t nsteps)
{
    size_t nn = nn3(s);
    for (int it = 0; it < nsteps; it++) {
        for (int f = 0; f < 3; f++) memset(s->J[f], 0, sizeof(int64_t) * nn);
        for (int sp = 0; sp < s->nsp; sp++) {
            int64_t n = s->np[sp];
            size_t b = sizeof(double) * (n ? n : 1);
            double *x0 = malloc(b), *y0 = malloc(b), *z0 = malloc(b);
            memcpy(x0, s->x[sp], b); memcpy(y0, s->y[sp], b); memcpy(z0, s->z[sp], b);
            for (int64_t p = 0; p < n; p++) push_particle3(s, sp, p);
            if (s->c.mode == 0)
                oracle3_deposit_current(s->c.nx, s->c.ny, s->c.nz, n, s->q[sp] > 0 ? 1 : -1, x0, y0, z0, s->x[sp], s->y[sp],
                                        s->z[sp], s->J[0], s->J[1], s->J[2]);
            free(x0); free(y0); free(z0);
        }
        redeposit3(s);
        if (s->c.mode == 0) oracle3_maxwell(s);
        s->step++;
    }
}

void oracle3_energy(const ostate3* s, double out[5])
{
    for (int i = 0; i < 5; i++) out[i] = 0.0;
    for (int sp = 0; sp < s->nsp; sp++) {
        double acc = 0.0;
        for (int64_t p = 0; p < s->np[sp]; p++) {
            double u2 = s->ux[sp][p] * s->ux[sp][p] + s->uy[sp][p] * s->uy[sp][p] + s->uz[sp][p] * s->uz[sp][p];
            acc += u2 / (sqrt(1.0 + u2) + 1.0);
        }
        out[sp] = acc * s->w * s->m[sp] * O_C * O_C;
    }
    int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    double vol = s->c.dx * s->c.dx * s->c.dx, mu0 = 1.0 / (O_EPS0 * O_C * O_C), eE = 0.0, eB = 0.0;
    for (int k = 0; k <= nz; k++) {
        double wn = (k == 0 || k == nz) ? 0.5 : 1.0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = N3(s, i, j, k);
                eE += wn * (s->F[0][c] * s->F[0][c] + s->F[1][c] * s->F[1][c]);
                eB += wn * s->F[5][c] * s->F[5][c];
                if (k < nz) {
                    eE += s->F[2][c] * s->F[2][c];
                    eB += s->F[3][c] * s->F[3][c] + s->F[4][c] * s->F[4][c];
                }
            }
    }
    out[2] = 0.5 * O_EPS0 * eE * vol;
    out[3] = 0.5 / mu0 * eB * vol;
    double pe = 0.0;
    for (int64_t p = 0; p < s->np[0]; p++) {
        double F[3], e;
        pair_force3_at(s, s->x[0][p], s->y[0][p], s->z[0][p], F, &e);
        pe += e;
    }
    out[4] = pe * s->w;
}

/* ======================================================================================== */
/* Differentiable transport stage (2D, neutral atoms, pair force only) with continuous       */
/* deposition (no fixed point) and its exact reverse-mode adjoint, in FP64.                 */
/* Loss L = sum_nodes cw(node) n^(node) at the final step + kin * (total kinetic energy).   */
/* Gradients with respect to D and r0 (r0 enters the force scale D/r0, Eq. (1)'s r0/dx and  */
/* the density unit n0 = r0^-3).                                                              */
/* ======================================================================================== */

/* continuous node density in units of n0, wall rows doubled */
static void dens_cont(const ostate* s, const double* x, const double* z, int64_t n, double* nh)
{
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    memset(nh, 0, sizeof(double) * nn);
    double unit = s->w / (s->c.dx * s->c.dx) * pow(s->r0, 3.0);
    for (int64_t p = 0; p < n; p++) {
        int64_t i = (int64_t)floor(x[p]), k = (int64_t)floor(z[p]);
        double fx = x[p] - i, fz = z[p] - k;
        if (k >= nz) { k = nz - 1; fz = 1.0; }
        double wx[2] = {1 - fx, fx}, wz[2] = {1 - fz, fz};
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) nh[(size_t)(k + b) * nx + imod(i + a, nx)] += unit * wx[a] * wz[b];
    }
    for (int i = 0; i < nx; i++) { nh[i] *= 2.0; nh[(size_t)nz * nx + i] *= 2.0; }
}

/* bilinear density, gradient and the mixed second derivative at (x, z) from a node array */
static void gather_cont(const ostate* s, const double* nh, double x, double z, double* n, double* gx, double* gz,
                        double* gxz, int64_t* ci, int64_t* ck, double* cfx, double* cfz)
{
    int nx = s->c.nx, nz = s->c.nz;
    int64_t i = (int64_t)floor(x), k = (int64_t)floor(z);
    double fx = x - i, fz = z - k;
    if (k >= nz) { k = nz - 1; fz = 1.0; }
    double n00 = nh[(size_t)k * nx + imod(i, nx)], n10 = nh[(size_t)k * nx + imod(i + 1, nx)];
    double n01 = nh[(size_t)(k + 1) * nx + imod(i, nx)], n11 = nh[(size_t)(k + 1) * nx + imod(i + 1, nx)];
    *n = (1 - fx) * (1 - fz) * n00 + fx * (1 - fz) * n10 + (1 - fx) * fz * n01 + fx * fz * n11;
    *gx = (1 - fz) * (n10 - n00) + fz * (n11 - n01);
    *gz = (1 - fx) * (n01 - n00) + fx * (n11 - n10);
    *gxz = n11 - n01 - n10 + n00;
    *ci = i; *ck = k; *cfx = fx; *cfz = fz;
}

/* Force along one axis (N) and its partial derivatives, Eqs. (1)-(3):
 * F = (D/r0)[U'(a) - U'(b)], a = rbar/(1-h), b = rbar/(1+h), rbar = n^(-1/3),
 * h = -(1/6)(r0/dx) n^(-4/3) q.  Outputs dF/dn, dF/dq and dF/dr0 at fixed (n, q). */
static double axis_force_d(double n, double q, double D, double r0, double dx, double* dFdn, double* dFdq, double* dFdr0)
{
    *dFdn = *dFdq = *dFdr0 = 0.0;
    if (!(n > 0.0)) return 0.0;
    double rbar = pow(n, -1.0 / 3.0);
    double h = -(1.0 / 6.0) * (r0 / dx) * pow(n, -4.0 / 3.0) * q;
    double drbar_dn = -(1.0 / 3.0) * pow(n, -4.0 / 3.0);
    double dh_dn = (2.0 / 9.0) * (r0 / dx) * pow(n, -7.0 / 3.0) * q;
    double dh_dq = -(1.0 / 6.0) * (r0 / dx) * pow(n, -4.0 / 3.0);
    double dh_dr0 = h / r0;
    double fu = D / r0, F = 0.0, dF_drbar = 0.0, dF_dh = 0.0;
    if (1.0 - h > 0.0) {
        double a = rbar / (1.0 - h);
        double up = oracle_lj_dU(a), upp = (156.0 * pow(a, -14.0) - 84.0 * pow(a, -8.0));
        F += fu * up;
        dF_drbar += fu * upp / (1.0 - h);
        dF_dh += fu * upp * rbar / ((1.0 - h) * (1.0 - h));
    }
    if (1.0 + h > 0.0) {
        double b = rbar / (1.0 + h);
        double up = oracle_lj_dU(b), upp = (156.0 * pow(b, -14.0) - 84.0 * pow(b, -8.0));
        F -= fu * up;
        dF_drbar -= fu * upp / (1.0 + h);
        dF_dh += fu * upp * rbar / ((1.0 + h) * (1.0 + h));
    }
    *dFdn = dF_drbar * drbar_dn + dF_dh * dh_dn;
    *dFdq = dF_dh * dh_dq;
    *dFdr0 = -F / r0 + dF_dh * dh_dr0;
    return F;
}

/* one forward transport step with continuous deposition; positions in cells, u = gamma v / c */
static void transport_step_cont(ostate* s, double* x, double* z, double* ux, double* uy, double* uz, int64_t n,
                                double* nh, int* refl)
{
    dens_cont(s, x, z, n, nh);
    double kick = s->dt / (s->m[0] * O_C);
    for (int64_t p = 0; p < n; p++) {
        double nn_, gx, gz, gxz, fx, fz; int64_t i, k;
        gather_cont(s, nh, x[p], z[p], &nn_, &gx, &gz, &gxz, &i, &k, &fx, &fz);
        double d1, d2, d3;
        double Fx = axis_force_d(nn_, gx, s->D, s->r0, s->c.dx, &d1, &d2, &d3);
        double Fz = axis_force_d(nn_, gz, s->D, s->r0, s->c.dx, &d1, &d2, &d3);
        ux[p] += kick * Fx;
        uz[p] += kick * Fz;
        double g = sqrt(1.0 + ux[p] * ux[p] + uy[p] * uy[p] + uz[p] * uz[p]);
        double step = O_C * s->dt / (g * s->c.dx);
        x[p] += ux[p] * step;
        z[p] += uz[p] * step;
        if (x[p] < 0.0) x[p] += s->c.nx;
        if (x[p] >= s->c.nx) x[p] -= s->c.nx;
        refl[p] = 0;
        if (z[p] < 0.0) { z[p] = -z[p]; uz[p] = -uz[p]; refl[p] = 1; }
        if (z[p] >= s->c.nz) { z[p] = 2.0 * s->c.nz - z[p]; uz[p] = -uz[p]; refl[p] = 1; }
    }
}

/* Adds to lx, lz the derivative of sum_nodes lam(node) nh(node) with respect to each particle's
 * position (the transpose of the deposition), lam in units of 1 / n0. */
static void deposit_transpose(const ostate* s, const double* lam, const double* x, const double* z, int64_t n,
                              double* lx, double* lz)
{
    int nx = s->c.nx, nz = s->c.nz;
    double unit = s->w / (s->c.dx * s->c.dx) * pow(s->r0, 3.0);
    for (int64_t p = 0; p < n; p++) {
        int64_t i = (int64_t)floor(x[p]), k = (int64_t)floor(z[p]);
        double fx = x[p] - i, fz = z[p] - k;
        if (k >= nz) { k = nz - 1; fz = 1.0; }
        double m0 = (k == 0) ? 2.0 : 1.0, m1 = (k + 1 == nz) ? 2.0 : 1.0;
        double l00 = m0 * lam[(size_t)k * nx + imod(i, nx)], l10 = m0 * lam[(size_t)k * nx + imod(i + 1, nx)];
        double l01 = m1 * lam[(size_t)(k + 1) * nx + imod(i, nx)], l11 = m1 * lam[(size_t)(k + 1) * nx + imod(i + 1, nx)];
        lx[p] += unit * ((1 - fz) * (l10 - l00) + fz * (l11 - l01));
        lz[p] += unit * ((1 - fx) * (l01 - l00) + fx * (l11 - l10));
    }
}

/* Forward nsteps from the current state (continuous deposition), loss and its gradient.
 * cw: node weights of the crater functional ((nz+1)*nx, units 1/n0), kin: weight of the kinetic
 * energy (1/J). out[0] = L, out[1] = dL/dD (1/J), out[2] = dL/dr0 (1/m). The state is advanced. */
void oracle_transport_grad(ostate* s, int32_t nsteps, const double* cw, double kin, double* out)
{
    int64_t n = s->np[0];
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    double *X = malloc(sizeof(double) * n * (nsteps + 1)), *Z = malloc(sizeof(double) * n * (nsteps + 1));
    double *UX = malloc(sizeof(double) * n * (nsteps + 1)), *UY = malloc(sizeof(double) * n * (nsteps + 1));
    double *UZ = malloc(sizeof(double) * n * (nsteps + 1));
    int* RF = malloc(sizeof(int) * (size_t)n * (nsteps > 0 ? nsteps : 1));
    double* nh = malloc(sizeof(double) * nn);
    memcpy(X, s->x[0], sizeof(double) * n); memcpy(Z, s->z[0], sizeof(double) * n);
    memcpy(UX, s->ux[0], sizeof(double) * n); memcpy(UY, s->uy[0], sizeof(double) * n); memcpy(UZ, s->uz[0], sizeof(double) * n);
    for (int t = 0; t < nsteps; t++) {
        double *x = X + (size_t)(t + 1) * n, *z = Z + (size_t)(t + 1) * n;
        double *ux = UX + (size_t)(t + 1) * n, *uy = UY + (size_t)(t + 1) * n, *uz = UZ + (size_t)(t + 1) * n;
        memcpy(x, X + (size_t)t * n, sizeof(double) * n); memcpy(z, Z + (size_t)t * n, sizeof(double) * n);
        memcpy(ux, UX + (size_t)t * n, sizeof(double) * n); memcpy(uy, UY + (size_t)t * n, sizeof(double) * n);
        memcpy(uz, UZ + (size_t)t * n, sizeof(double) * n);
        transport_step_cont(s, x, z, ux, uy, uz, n, nh, RF + (size_t)t * n);
    }
    /* loss */
    double *xN = X + (size_t)nsteps * n, *zN = Z + (size_t)nsteps * n;
    double *uxN = UX + (size_t)nsteps * n, *uyN = UY + (size_t)nsteps * n, *uzN = UZ + (size_t)nsteps * n;
    dens_cont(s, xN, zN, n, nh);
    double L = 0.0;
    for (size_t c = 0; c < nn; c++) L += cw[c] * nh[c];
    double mc2w = s->w * s->m[0] * O_C * O_C, ke = 0.0;
    for (int64_t p = 0; p < n; p++) {
        double u2 = uxN[p] * uxN[p] + uyN[p] * uyN[p] + uzN[p] * uzN[p];
        ke += mc2w * u2 / (sqrt(1.0 + u2) + 1.0);
    }
    L += kin * ke;
    /* adjoint seeds: lambda_x = transpose of the final deposition; lambda_u = kin * w m c^2 u / gamma */
    double *lx = calloc(n, sizeof(double)), *lz = calloc(n, sizeof(double));
    double *lux = calloc(n, sizeof(double)), *luy = calloc(n, sizeof(double)), *luz = calloc(n, sizeof(double));
    double* lam = malloc(sizeof(double) * nn);
    deposit_transpose(s, cw, xN, zN, n, lx, lz);
    /* The r0 dependence of the final density (n0 = r0^-3 scales every node): dn^/dr0 = 3 n^/r0 */
    double gD = 0.0, gr0 = 0.0;
    for (size_t c = 0; c < nn; c++) gr0 += cw[c] * 3.0 * nh[c] / s->r0;
    for (int64_t p = 0; p < n; p++) {
        double u2 = uxN[p] * uxN[p] + uyN[p] * uyN[p] + uzN[p] * uzN[p], g = sqrt(1.0 + u2);
        lux[p] = kin * mc2w * uxN[p] / g; luy[p] = kin * mc2w * uyN[p] / g; luz[p] = kin * mc2w * uzN[p] / g;
    }
    double kick = s->dt / (s->m[0] * O_C);
    for (int t = nsteps - 1; t >= 0; t--) {
        double *x0 = X + (size_t)t * n, *z0 = Z + (size_t)t * n;
        double *ux1 = UX + (size_t)(t + 1) * n, *uy1 = UY + (size_t)(t + 1) * n, *uz1 = UZ + (size_t)(t + 1) * n;
        int* rf = RF + (size_t)t * n;
        dens_cont(s, x0, z0, n, nh);
        memset(lam, 0, sizeof(double) * nn);
        for (int64_t p = 0; p < n; p++) {
            /* position update: x1 = x0 + c dt u / (gamma dx) (then the wall mirror) */
            double lzp = lz[p], luzp = luz[p];
            double ux = ux1[p], uy = uy1[p], uz = uz1[p];
            if (rf[p]) { lzp = -lzp; luzp = -luzp; uz = -uz; }   /* undo the mirror: z1 = -z', u_z1 = -u_z' */
            double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz), cs = O_C * s->dt / (s->c.dx * g);
            double lu[3] = {lux[p], luy[p], luzp};
            double u[3] = {ux, uy, uz}, lp[3] = {lx[p], 0.0, lzp};
            double udl = (u[0] * lp[0] + u[2] * lp[2]) / (g * g);
            for (int d = 0; d < 3; d++) lu[d] += cs * (lp[d] - u[d] * udl);
            /* kick: u' = u + kick F(x0): lambda_u unchanged backwards, lambda_F = kick lambda_u */
            double nn_, gx, gz, gxz, fx, fz; int64_t i, k;
            gather_cont(s, nh, x0[p], z0[p], &nn_, &gx, &gz, &gxz, &i, &k, &fx, &fz);
            double dxn, dxq, dxr, dzn, dzq, dzr;
            double Fx = axis_force_d(nn_, gx, s->D, s->r0, s->c.dx, &dxn, &dxq, &dxr);
            double Fz = axis_force_d(nn_, gz, s->D, s->r0, s->c.dx, &dzn, &dzq, &dzr);
            double lFx = kick * lu[0], lFz = kick * lu[2];
            gD += (lFx * Fx + lFz * Fz) / s->D;
            /* r0: explicit part, and the n0 = r0^-3 scaling of n and q (both proportional to r0^3) */
            gr0 += lFx * (dxr + dxn * 3.0 * nn_ / s->r0 + dxq * 3.0 * gx / s->r0);
            gr0 += lFz * (dzr + dzn * 3.0 * nn_ / s->r0 + dzq * 3.0 * gz / s->r0);
            double ln = lFx * dxn + lFz * dzn, lqx = lFx * dxq, lqz = lFz * dzq;
            /* gather: n = bilinear, q_x = d/dxi, q_z = d/dzeta; their position derivatives */
            lx[p] = lp[0] + ln * gx + lqx * 0.0 + lqz * gxz;
            lz[p] = lp[2] + ln * gz + lqx * gxz + lqz * 0.0;
            lux[p] = lu[0]; luy[p] = lu[1]; luz[p] = lu[2];
            /* transpose of the gather onto the nodes */
            double w00 = (1 - fx) * (1 - fz), w10 = fx * (1 - fz), w01 = (1 - fx) * fz, w11 = fx * fz;
            size_t c00 = (size_t)k * nx + imod(i, nx), c10 = (size_t)k * nx + imod(i + 1, nx);
            size_t c01 = (size_t)(k + 1) * nx + imod(i, nx), c11 = (size_t)(k + 1) * nx + imod(i + 1, nx);
            lam[c00] += ln * w00 + lqx * (-(1 - fz)) + lqz * (-(1 - fx));
            lam[c10] += ln * w10 + lqx * (1 - fz) + lqz * (-fx);
            lam[c01] += ln * w01 + lqx * (-fz) + lqz * (1 - fx);
            lam[c11] += ln * w11 + lqx * fz + lqz * fx;
        }
        /* the nodes depend on every particle's position: transpose of the deposition */
        deposit_transpose(s, lam, x0, z0, n, lx, lz);
        /* and on r0 through n0 = r0^-3 (already counted in the force terms above) */
    }
    out[0] = L; out[1] = gD; out[2] = gr0;
    /* leave the final state in the context */
    memcpy(s->x[0], xN, sizeof(double) * n); memcpy(s->z[0], zN, sizeof(double) * n);
    memcpy(s->ux[0], uxN, sizeof(double) * n); memcpy(s->uy[0], uyN, sizeof(double) * n); memcpy(s->uz[0], uzN, sizeof(double) * n);
    free(X); free(Z); free(UX); free(UY); free(UZ); free(RF); free(nh); free(lx); free(lz); free(lux); free(luy); free(luz); free(lam);
}

/* Loss of the same functional after nsteps forward (continuous deposition), no gradient: for
 * finite differences. D and r0 override the configuration's values for this call. */
double oracle_transport_loss(ostate* s, int32_t nsteps, const double* cw, double kin, double D_J, double r0_m)
{
    int64_t n = s->np[0];
    double Dsave = s->D, r0save = s->r0;
    s->D = D_J; s->r0 = r0_m;
    double *x = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *ux = malloc(sizeof(double) * n), *uy = malloc(sizeof(double) * n), *uz = malloc(sizeof(double) * n);
    int* rf = malloc(sizeof(int) * (n ? n : 1));
    memcpy(x, s->x[0], sizeof(double) * n); memcpy(z, s->z[0], sizeof(double) * n);
    memcpy(ux, s->ux[0], sizeof(double) * n); memcpy(uy, s->uy[0], sizeof(double) * n); memcpy(uz, s->uz[0], sizeof(double) * n);
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    double* nh = malloc(sizeof(double) * nn);
    for (int t = 0; t < nsteps; t++) transport_step_cont(s, x, z, ux, uy, uz, n, nh, rf);
    dens_cont(s, x, z, n, nh);
    double L = 0.0, mc2w = s->w * s->m[0] * O_C * O_C;
    for (size_t c = 0; c < nn; c++) L += cw[c] * nh[c];
    for (int64_t p = 0; p < n; p++) {
        double u2 = ux[p] * ux[p] + uy[p] * uy[p] + uz[p] * uz[p];
        L += kin * mc2w * u2 / (sqrt(1.0 + u2) + 1.0);
    }
    s->D = Dsave; s->r0 = r0save;
    free(x); free(z); free(ux); free(uy); free(uz); free(rf); free(nh);
    return L;
}

double oracle_D(const ostate* s) { return s->D; }
double oracle_r0(const ostate* s) { return s->r0; }

/* ======================================================================================== */
/* Differentiable full cycle (2D: ions, electrons, fields, laser) with continuous            */
/* deposition (linear weights of the unrounded positions, no fixed point) and its exact      */
/* reverse mode, in FP64.                                                                     */
/* Loss L = sum_nodes cw(node) n^(node) of the final ion density + kin * (total kinetic       */
/* energy of all species). Gradients with respect to D, r0 (pair potential, Eqs. 1-3) and    */
/* the peak intensity I0 (E0 = sqrt(2 I0 / (eps0 c)) scales the antenna source).              */
/*                                                                                            */
/* One forward step from the state (X, U, F) at step t:                                       */
/*   n^ = dens(X_ions); per particle: E, B gathered at x, pair force F_p(n^) for ions,        */
/*   Boris -> u', x' = x + c dt u'/(gamma' dx), walls; current j = J(x, x', u'_y/gamma');     */
/*   Maxwell: B += H E (half), E = M(E, B, j) with Mur walls and the antenna, B += H E (half).*/
/* j is held as the scaled arrays dt J / eps0 that the E update subtracts.                   */
/* ======================================================================================== */

static double hat_c(double d) { double a = fabs(d); return a < 1.0 ? 1.0 - a : 0.0; }
static double dhat_c(double d) { return fabs(d) < 1.0 ? (d > 0.0 ? -1.0 : 1.0) : 0.0; }

/* dt J / eps0 per unit of the continuous Esirkepov sums (2 Wx, 6 Wy beta, 2 Wz) */
static double cur_cx(const ostate* s) { return O_QE * s->w / (2.0 * s->c.dx * O_EPS0); }
static double cur_cy(const ostate* s) { return O_QE * s->w * O_C * s->dt / (6.0 * s->c.dx * s->c.dx * O_EPS0); }

/* Esirkepov current (linear weights) of one particle moving (x0, z0) -> (x1, z1) (x1 unwrapped
 * to within half a period of x0, z1 after the wall mirror), with beta_y = by; sg = charge sign. */
static void cur_cont(const ostate* s, double sg, double x0, double z0, double x1, double z1, double by,
                     double* jx, double* jy, double* jz)
{
    int nx = s->c.nx, nz = s->c.nz;
    double bx = floor(x0 < x1 ? x0 : x1), bz = floor(z0 < z1 ? z0 : z1);
    double S0x[3], S1x[3], S0z[3], S1z[3];
    for (int a = 0; a < 3; a++) {
        S0x[a] = hat_c(x0 - (bx + a)); S1x[a] = hat_c(x1 - (bx + a));
        S0z[a] = hat_c(z0 - (bz + a)); S1z[a] = hat_c(z1 - (bz + a));
    }
    double cx = sg * cur_cx(s), cy = sg * cur_cy(s) * by;
    int64_t ib = (int64_t)bx, kb = (int64_t)bz;
    for (int b = 0; b < 3; b++) {
        int64_t l = kb + b;
        if (l > nz) continue;                        /* weights there are zero */
        double acc = 0.0;
        for (int a = 0; a < 2; a++) {
            acc -= (S1x[a] - S0x[a]) * (S0z[b] + S1z[b]);
            jx[(size_t)l * nx + imod(ib + a, nx)] += cx * acc;
        }
        for (int a = 0; a < 3; a++)
            jy[(size_t)l * nx + imod(ib + a, nx)] +=
                cy * (2 * S0x[a] * S0z[b] + S1x[a] * S0z[b] + S0x[a] * S1z[b] + 2 * S1x[a] * S1z[b]);
    }
    for (int a = 0; a < 3; a++) {
        double acc = 0.0;
        for (int b = 0; b < 2; b++) {
            int64_t l = kb + b;
            acc -= (S1z[b] - S0z[b]) * (S0x[a] + S1x[a]);
            if (l <= nz) jz[(size_t)l * nx + imod(ib + a, nx)] += cur_cx(s) * sg * acc;
        }
    }
}

/* Transpose of cur_cont: with node adjoints lj (of jx, jy, jz), adds d/d(x0, z0, x1, z1, by) of
 * sum lj * j into g[0..4]. */
static void cur_cont_T(const ostate* s, double sg, double x0, double z0, double x1, double z1, double by,
                       const double* ljx, const double* ljy, const double* ljz, double g[5])
{
    int nx = s->c.nx, nz = s->c.nz;
    double bx = floor(x0 < x1 ? x0 : x1), bz = floor(z0 < z1 ? z0 : z1);
    int64_t ib = (int64_t)bx, kb = (int64_t)bz;
    double S0x[3], S1x[3], S0z[3], S1z[3];
    for (int a = 0; a < 3; a++) {
        S0x[a] = hat_c(x0 - (bx + a)); S1x[a] = hat_c(x1 - (bx + a));
        S0z[a] = hat_c(z0 - (bz + a)); S1z[a] = hat_c(z1 - (bz + a));
    }
    double Lx[3][3], Ly[3][3], Lz[3][3];              /* [a][b] */
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            int64_t l = kb + b;
            size_t c = (size_t)l * nx + imod(ib + a, nx);
            Lx[a][b] = l <= nz ? ljx[c] : 0.0;
            Ly[a][b] = l <= nz ? ljy[c] : 0.0;
            Lz[a][b] = l <= nz ? ljz[c] : 0.0;
        }
    double cx = sg * cur_cx(s), cy = sg * cur_cy(s);
    double dS0x[3] = {0, 0, 0}, dS1x[3] = {0, 0, 0}, dS0z[3] = {0, 0, 0}, dS1z[3] = {0, 0, 0};
    /* x current: value = cx sum_b (S0z+S1z)[b] * (-sum_{a<=1} dSx[a] Rx[a][b]),
     * Rx[a][b] = sum_{a' = a..1} Lx[a'][b] */
    for (int b = 0; b < 3; b++) {
        double Rx1 = Lx[1][b], Rx0 = Lx[0][b] + Lx[1][b];
        double zsum = S0z[b] + S1z[b];
        double dx0 = S1x[0] - S0x[0], dx1 = S1x[1] - S0x[1];
        dS1x[0] += -cx * zsum * Rx0; dS0x[0] += cx * zsum * Rx0;
        dS1x[1] += -cx * zsum * Rx1; dS0x[1] += cx * zsum * Rx1;
        double zz = -cx * (dx0 * Rx0 + dx1 * Rx1);
        dS0z[b] += zz; dS1z[b] += zz;
    }
    /* z current */
    for (int a = 0; a < 3; a++) {
        double Rz1 = Lz[a][1], Rz0 = Lz[a][0] + Lz[a][1];
        double xsum = S0x[a] + S1x[a];
        double dz0 = S1z[0] - S0z[0], dz1 = S1z[1] - S0z[1];
        dS1z[0] += -cx * xsum * Rz0; dS0z[0] += cx * xsum * Rz0;
        dS1z[1] += -cx * xsum * Rz1; dS0z[1] += cx * xsum * Rz1;
        double xx = -cx * (dz0 * Rz0 + dz1 * Rz1);
        dS0x[a] += xx; dS1x[a] += xx;
    }
    /* y current: value = cy by sum Ly w6 */
    double gby = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double L = Ly[a][b] * cy;
            gby += L * (2 * S0x[a] * S0z[b] + S1x[a] * S0z[b] + S0x[a] * S1z[b] + 2 * S1x[a] * S1z[b]);
            dS0x[a] += by * L * (2 * S0z[b] + S1z[b]);
            dS1x[a] += by * L * (S0z[b] + 2 * S1z[b]);
            dS0z[b] += by * L * (2 * S0x[a] + S1x[a]);
            dS1z[b] += by * L * (S0x[a] + 2 * S1x[a]);
        }
    for (int a = 0; a < 3; a++) {
        g[0] += dS0x[a] * dhat_c(x0 - (bx + a));
        g[1] += dS0z[a] * dhat_c(z0 - (bz + a));
        g[2] += dS1x[a] * dhat_c(x1 - (bx + a));
        g[3] += dS1z[a] * dhat_c(z1 - (bz + a));
    }
    g[4] += gby;
}

/* Yee half step of B from E (the arrays of one state) */
static void hb_cont(const ostate* s, double* F)
{
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    double h = 0.5 * s->dt / s->c.dx;
    double *Ex = F, *Ey = F + nn, *Ez = F + 2 * nn, *Bx = F + 3 * nn, *By = F + 4 * nn, *Bz = F + 5 * nn;
    for (int k = 0; k <= nz; k++)
        for (int i = 0; i < nx; i++) {
            int ip = (i + 1) % nx;
            size_t c = (size_t)k * nx + i;
            if (k < nz) {
                Bx[c] += h * (Ey[c + nx] - Ey[c]);
                By[c] += h * ((Ez[(size_t)k * nx + ip] - Ez[c]) - (Ex[c + nx] - Ex[c]));
            }
            Bz[c] -= h * (Ey[(size_t)k * nx + ip] - Ey[c]);
        }
}

/* transpose of hb_cont: lamE += H^T lamB (lamB unchanged) */
static void hb_cont_T(const ostate* s, double* lF)
{
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    double h = 0.5 * s->dt / s->c.dx;
    double *lEx = lF, *lEy = lF + nn, *lEz = lF + 2 * nn, *lBx = lF + 3 * nn, *lBy = lF + 4 * nn, *lBz = lF + 5 * nn;
    for (int k = 0; k <= nz; k++)
        for (int i = 0; i < nx; i++) {
            int ip = (i + 1) % nx;
            size_t c = (size_t)k * nx + i;
            if (k < nz) {
                lEy[c + nx] += h * lBx[c]; lEy[c] -= h * lBx[c];
                lEz[(size_t)k * nx + ip] += h * lBy[c]; lEz[c] -= h * lBy[c];
                lEx[c + nx] -= h * lBy[c]; lEx[c] += h * lBy[c];
            }
            lEy[(size_t)k * nx + ip] -= h * lBz[c]; lEy[c] += h * lBz[c];
        }
}

/* laser source per unit E0 (E_x of the incident pulse at x, t divided by E0) */
static double laser_shape(ostate* s, double x_cells, double t)
{
    double save = s->E0;
    s->E0 = 1.0;
    double v = laser_field(s, x_cells, t);
    s->E0 = save;
    return v;
}

/* E update of the Yee scheme with Mur walls and the antenna (E0 given), j = dt J / eps0 */
static void fe_cont(ostate* s, double* F, const double* jx, const double* jy, const double* jz, double E0, double tmid)
{
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    double cdt = O_C * s->dt, h = O_C * O_C * s->dt / s->c.dx;
    double *Ex = F, *Ey = F + nn, *Ez = F + 2 * nn, *Bx = F + 3 * nn, *By = F + 4 * nn, *Bz = F + 5 * nn;
    double* nEx = malloc(sizeof(double) * nn);
    double* nEy = malloc(sizeof(double) * nn);
    for (int k = 0; k <= nz; k++)
        for (int i = 0; i < nx; i++) {
            int im = (i + nx - 1) % nx;
            size_t c = (size_t)k * nx + i;
            nEx[c] = Ex[c];
            nEy[c] = Ey[c];
            if (k > 0 && k < nz) {
                nEx[c] = Ex[c] - h * (By[c] - By[c - nx]) - jx[c];
                nEy[c] = Ey[c] + h * ((Bx[c] - Bx[c - nx]) - (Bz[c] - Bz[(size_t)k * nx + im])) - jy[c];
                if (k == s->k_ant) nEx[c] += 2.0 * (cdt / s->c.dx) * E0 * laser_shape(s, (double)i + 0.5, tmid);
            }
        }
    double alpha = (cdt - s->c.dx) / (cdt + s->c.dx);
    for (int i = 0; i < nx; i++) {
        size_t b0 = i, b1 = (size_t)nx + i, t0 = (size_t)nz * nx + i, t1 = (size_t)(nz - 1) * nx + i;
        nEx[b0] = Ex[b1] + alpha * (nEx[b1] - Ex[b0]);
        nEy[b0] = Ey[b1] + alpha * (nEy[b1] - Ey[b0]);
        nEx[t0] = Ex[t1] + alpha * (nEx[t1] - Ex[t0]);
        nEy[t0] = Ey[t1] + alpha * (nEy[t1] - Ey[t0]);
    }
    for (int k = 0; k < nz; k++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)k * nx + i;
            Ez[c] += h * (By[c] - By[(size_t)k * nx + (i + nx - 1) % nx]) - jz[c];
        }
    memcpy(Ex, nEx, sizeof(double) * nn);
    memcpy(Ey, nEy, sizeof(double) * nn);
    free(nEx); free(nEy);
}

/* Transpose of fe_cont. lF holds the adjoints of the new E (and of B, unchanged by this part);
 * on return it holds those of the old E and of B, lj the adjoints of jx, jy, jz, and *gE0 has
 * the derivative with respect to E0 added. */
static void fe_cont_T(ostate* s, double* lF, double* ljx, double* ljy, double* ljz, double tmid, double* gE0)
{
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    double cdt = O_C * s->dt, h = O_C * O_C * s->dt / s->c.dx;
    double *lEx = lF, *lEy = lF + nn, *lEz = lF + 2 * nn, *lBx = lF + 3 * nn, *lBy = lF + 4 * nn, *lBz = lF + 5 * nn;
    double* lnEx = malloc(sizeof(double) * nn);
    double* lnEy = malloc(sizeof(double) * nn);
    memcpy(lnEx, lEx, sizeof(double) * nn);
    memcpy(lnEy, lEy, sizeof(double) * nn);
    memset(lEx, 0, sizeof(double) * nn);
    memset(lEy, 0, sizeof(double) * nn);
    memset(ljx, 0, sizeof(double) * nn);
    memset(ljy, 0, sizeof(double) * nn);
    memset(ljz, 0, sizeof(double) * nn);
    /* Ez (in place): old Ez passes through; B and jz receive */
    for (int k = 0; k < nz; k++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)k * nx + i;
            double v = lEz[c];
            lBy[c] += h * v;
            lBy[(size_t)k * nx + (i + nx - 1) % nx] -= h * v;
            ljz[c] = -v;
        }
    /* Mur rows (they overwrite the wall values of the new E) */
    double alpha = (cdt - s->c.dx) / (cdt + s->c.dx);
    for (int i = 0; i < nx; i++) {
        size_t b0 = i, b1 = (size_t)nx + i, t0 = (size_t)nz * nx + i, t1 = (size_t)(nz - 1) * nx + i;
        double v;
        v = lnEx[b0]; lEx[b1] += v; lnEx[b1] += alpha * v; lEx[b0] -= alpha * v; lnEx[b0] = 0.0;
        v = lnEy[b0]; lEy[b1] += v; lnEy[b1] += alpha * v; lEy[b0] -= alpha * v; lnEy[b0] = 0.0;
        v = lnEx[t0]; lEx[t1] += v; lnEx[t1] += alpha * v; lEx[t0] -= alpha * v; lnEx[t0] = 0.0;
        v = lnEy[t0]; lEy[t1] += v; lnEy[t1] += alpha * v; lEy[t0] -= alpha * v; lnEy[t0] = 0.0;
    }
    for (int k = 1; k < nz; k++)
        for (int i = 0; i < nx; i++) {
            int im = (i + nx - 1) % nx;
            size_t c = (size_t)k * nx + i;
            double v = lnEx[c];
            lEx[c] += v;
            lBy[c] -= h * v;
            lBy[c - nx] += h * v;
            ljx[c] = -v;
            if (k == s->k_ant) *gE0 += v * 2.0 * (cdt / s->c.dx) * laser_shape(s, (double)i + 0.5, tmid);
            v = lnEy[c];
            lEy[c] += v;
            lBx[c] += h * v;
            lBx[c - nx] -= h * v;
            lBz[c] -= h * v;
            lBz[(size_t)k * nx + im] += h * v;
            ljy[c] = -v;
        }
    free(lnEx); free(lnEy);
}

/* Maxwell part of one step on the arrays F (6 nn) with the scaled current j (3 nn) */
static void maxwell_cont(ostate* s, double* F, const double* j, double E0, int64_t step)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    hb_cont(s, F);
    fe_cont(s, F, j, j + nn, j + 2 * nn, E0, ((double)step + 0.5) * s->dt);
    hb_cont(s, F);
}

/* its transpose: lF (adjoint of the new fields) -> adjoint of the old fields; lj receives the
 * current's adjoint; *gE0 accumulates the E0 derivative */
static void maxwell_cont_T(ostate* s, double* lF, double* lj, int64_t step, double* gE0)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    hb_cont_T(s, lF);
    fe_cont_T(s, lF, lj, lj + nn, lj + 2 * nn, ((double)step + 0.5) * s->dt, gE0);
    hb_cont_T(s, lF);
}

void oracle_maxwell_cont(ostate* s, double* F, const double* j, double E0, int64_t step)
{
    maxwell_cont(s, F, j, E0, step);
}

void oracle_maxwell_cont_T(ostate* s, double* lF, double* lj, int64_t step, double* gE0)
{
    maxwell_cont_T(s, lF, lj, step, gE0);
}

/* staggered bilinear gather from an array (as gather_field) and its transpose: adds lv * weights
 * into lA and the position derivatives lv * dA/dx, lv * dA/dz into *lx, *lz */
static double gather_arr(const ostate* s, const double* A, double x, double z, double sx, double sz,
                         double* lA, double lv, double* lx, double* lz)
{
    int nx = s->c.nx, nz = s->c.nz;
    double xs = x - sx, zs = z - sz;
    int64_t rows = sz > 0 ? nz : nz + 1;
    int clamped = 0;
    if (zs < 0.0) { zs = 0.0; clamped = 1; }
    if (zs > (double)(rows - 1)) { zs = (double)(rows - 1); clamped = 1; }
    int64_t i = (int64_t)floor(xs), k = (int64_t)floor(zs);
    double fx = xs - (double)i, fz = zs - (double)k;
    if (k >= rows - 1) { k = rows - 2; fz = 1.0; }
    size_t c00 = (size_t)k * nx + imod(i, nx), c10 = (size_t)k * nx + imod(i + 1, nx);
    size_t c01 = c00 + nx, c11 = c10 + nx;
    double a00 = A[c00], a10 = A[c10], a01 = A[c01], a11 = A[c11];
    double v = (1 - fx) * (1 - fz) * a00 + fx * (1 - fz) * a10 + (1 - fx) * fz * a01 + fx * fz * a11;
    if (lA) {
        lA[c00] += lv * (1 - fx) * (1 - fz); lA[c10] += lv * fx * (1 - fz);
        lA[c01] += lv * (1 - fx) * fz;       lA[c11] += lv * fx * fz;
        *lx += lv * ((1 - fz) * (a10 - a00) + fz * (a11 - a01));
        if (!clamped) *lz += lv * ((1 - fx) * (a01 - a00) + fx * (a11 - a10));
    }
    return v;
}

static const double k_stag[6][2] = {{0.5, 0.0}, {0.0, 0.0}, {0.0, 0.5}, {0.0, 0.5}, {0.5, 0.5}, {0.5, 0.0}};

/* the intermediate values of one particle's forward step, kept for its transpose */
typedef struct {
    double E[3], B[3], Fp[3];
    double n, qx, qz, gxz, dxn, dxq, dxr, dzn, dzq, dzr;   /* pair-force pieces (ions) */
    double um[3], gm, tfac, t[3], t2, sv[3], upr[3], uf[3];
    double g, cs, xn, zn, x1u, z1, ufin[3], gfin, by;
    int refl;
} pstep;

static void particle_fwd(ostate* s, int sp, const double* F, const double* nh, double x, double z, const double u[3],
                         pstep* P)
{
    for (int d = 0; d < 3; d++) { P->E[d] = P->B[d] = P->Fp[d] = 0.0; }
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    if (s->c.mode == 0)
        for (int f = 0; f < 6; f++) {
            double v = gather_arr(s, F + f * nn, x, z, k_stag[f][0], k_stag[f][1], NULL, 0, NULL, NULL);
            if (f < 3) P->E[f] = v; else P->B[f - 3] = v;
        }
    if (s->pair[sp]) {
        int64_t i, k; double fx, fz;
        gather_cont(s, nh, x, z, &P->n, &P->qx, &P->qz, &P->gxz, &i, &k, &fx, &fz);
        P->Fp[0] = axis_force_d(P->n, P->qx, s->D, s->r0, s->c.dx, &P->dxn, &P->dxq, &P->dxr);
        P->Fp[2] = axis_force_d(P->n, P->qz, s->D, s->r0, s->c.dx, &P->dzn, &P->dzq, &P->dzr);
    }
    /* Boris, the steps of oracle_boris kept */
    double q = s->q[sp], m = s->m[sp], dt = s->dt;
    double eps = q * dt / (2.0 * m * O_C), fk = dt / (2.0 * m * O_C);
    for (int d = 0; d < 3; d++) P->um[d] = u[d] + eps * P->E[d] + fk * P->Fp[d];
    P->gm = sqrt(1.0 + P->um[0] * P->um[0] + P->um[1] * P->um[1] + P->um[2] * P->um[2]);
    P->tfac = q * dt / (2.0 * m * P->gm);
    for (int d = 0; d < 3; d++) P->t[d] = P->tfac * P->B[d];
    P->t2 = P->t[0] * P->t[0] + P->t[1] * P->t[1] + P->t[2] * P->t[2];
    for (int d = 0; d < 3; d++) P->sv[d] = 2.0 * P->t[d] / (1.0 + P->t2);
    const double* um = P->um; const double* t = P->t; const double* sv = P->sv;
    P->upr[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    P->upr[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    P->upr[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    double up[3];
    up[0] = um[0] + (P->upr[1] * sv[2] - P->upr[2] * sv[1]);
    up[1] = um[1] + (P->upr[2] * sv[0] - P->upr[0] * sv[2]);
    up[2] = um[2] + (P->upr[0] * sv[1] - P->upr[1] * sv[0]);
    for (int d = 0; d < 3; d++) P->uf[d] = up[d] + eps * P->E[d] + fk * P->Fp[d];
    /* move and walls */
    P->g = sqrt(1.0 + P->uf[0] * P->uf[0] + P->uf[1] * P->uf[1] + P->uf[2] * P->uf[2]);
    P->cs = O_C * dt / (P->g * s->c.dx);
    P->xn = x + P->uf[0] * P->cs;
    P->zn = z + P->uf[2] * P->cs;
    for (int d = 0; d < 3; d++) P->ufin[d] = P->uf[d];
    P->refl = 0;
    P->z1 = P->zn;
    if (P->zn < 0.0) { P->z1 = -P->zn; P->ufin[2] = -P->uf[2]; P->refl = 1; }
    if (P->zn >= s->c.nz) { P->z1 = 2.0 * s->c.nz - P->zn; P->ufin[2] = -P->uf[2]; P->refl = 1; }
    P->x1u = P->xn;                                 /* unwrapped: within a cell of x */
    P->gfin = P->g;
    P->by = P->ufin[1] / P->gfin;
}

static double wrap_x(const ostate* s, double x)
{
    if (x < 0.0) x += s->c.nx;
    if (x >= s->c.nx) x -= s->c.nx;
    return x;
}

/* one forward step of the continuous full cycle on the state arrays (positions, momenta of both
 * species, fields); j: scratch 3 nn; nh: scratch nn */
static void full_step_cont(ostate* s, double** X, double** Z, double** U, double* F, double* j, double* nh,
                           double E0, int64_t step)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    if (s->pair[0]) dens_cont(s, X[0], Z[0], s->np[0], nh);
    memset(j, 0, sizeof(double) * 3 * nn);
    for (int sp = 0; sp < s->nsp; sp++) {
        double sg = s->q[sp] > 0 ? 1.0 : (s->q[sp] < 0 ? -1.0 : 0.0);
        for (int64_t p = 0; p < s->np[sp]; p++) {
            pstep P;
            double* u = U[sp] + 3 * p;
            particle_fwd(s, sp, F, nh, X[sp][p], Z[sp][p], u, &P);
            if (s->c.mode == 0 && sg != 0.0)
                cur_cont(s, sg, X[sp][p], Z[sp][p], P.x1u, P.z1, P.by, j, j + nn, j + 2 * nn);
            X[sp][p] = wrap_x(s, P.xn);
            Z[sp][p] = P.z1;
            for (int d = 0; d < 3; d++) u[d] = P.ufin[d];
        }
    }
    if (s->c.mode == 0) maxwell_cont(s, F, j, E0, step);
}

/* kinetic energy of all species from packed momenta */
static double kinetic_all(const ostate* s, double** U)
{
    double ke = 0.0;
    for (int sp = 0; sp < s->nsp; sp++) {
        double acc = 0.0;
        for (int64_t p = 0; p < s->np[sp]; p++) {
            const double* u = U[sp] + 3 * p;
            double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            acc += u2 / (sqrt(1.0 + u2) + 1.0);
        }
        ke += acc * s->w * s->m[sp] * O_C * O_C;
    }
    return ke;
}

typedef struct {
    int nsteps;
    double *X[2], *Z[2], *U[2];     /* (nsteps + 1) * np each (U: 3 per particle) */
    double* F;                      /* (nsteps + 1) * 6 nn */
} ftraj;

static void traj_alloc(const ostate* s, ftraj* T, int nsteps)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    T->nsteps = nsteps;
    for (int sp = 0; sp < 2; sp++) {
        size_t n = sp < s->nsp ? (size_t)s->np[sp] : 0;
        T->X[sp] = malloc(sizeof(double) * (n ? n : 1) * (nsteps + 1));
        T->Z[sp] = malloc(sizeof(double) * (n ? n : 1) * (nsteps + 1));
        T->U[sp] = malloc(sizeof(double) * 3 * (n ? n : 1) * (nsteps + 1));
        for (size_t p = 0; p < n; p++) {
            T->X[sp][p] = s->x[sp][p]; T->Z[sp][p] = s->z[sp][p];
            T->U[sp][3 * p] = s->ux[sp][p]; T->U[sp][3 * p + 1] = s->uy[sp][p]; T->U[sp][3 * p + 2] = s->uz[sp][p];
        }
    }
    T->F = malloc(sizeof(double) * 6 * nn * (nsteps + 1));
    for (int f = 0; f < 6; f++) memcpy(T->F + f * nn, s->F[f], sizeof(double) * nn);
}

static void traj_free(ftraj* T)
{
    for (int sp = 0; sp < 2; sp++) { free(T->X[sp]); free(T->Z[sp]); free(T->U[sp]); }
    free(T->F);
}

/* run the stored trajectory forward; returns the loss of its final state */
static double traj_forward(ostate* s, ftraj* T, const double* cw, double kin, double E0)
{
    size_t nn = (size_t)s->c.nx * (s->c.nz + 1);
    double* j = malloc(sizeof(double) * 3 * nn);
    double* nh = malloc(sizeof(double) * nn);
    for (int t = 0; t < T->nsteps; t++) {
        double *X[2], *Z[2], *U[2];
        for (int sp = 0; sp < s->nsp; sp++) {
            size_t n = (size_t)s->np[sp];
            X[sp] = T->X[sp] + (t + 1) * n; Z[sp] = T->Z[sp] + (t + 1) * n; U[sp] = T->U[sp] + 3 * (t + 1) * n;
            memcpy(X[sp], T->X[sp] + t * n, sizeof(double) * n);
            memcpy(Z[sp], T->Z[sp] + t * n, sizeof(double) * n);
            memcpy(U[sp], T->U[sp] + 3 * t * n, sizeof(double) * 3 * n);
        }
        double* F = T->F + (size_t)(t + 1) * 6 * nn;
        memcpy(F, T->F + (size_t)t * 6 * nn, sizeof(double) * 6 * nn);
        full_step_cont(s, X, Z, U, F, j, nh, E0, s->step + t);
    }
    double L = 0.0;
    int N = T->nsteps;
    if (s->pair[0]) {
        dens_cont(s, T->X[0] + (size_t)N * s->np[0], T->Z[0] + (size_t)N * s->np[0], s->np[0], nh);
        for (size_t c = 0; c < nn; c++) L += cw[c] * nh[c];
    }
    double* UN[2];
    for (int sp = 0; sp < s->nsp; sp++) UN[sp] = T->U[sp] + 3 * (size_t)N * s->np[sp];
    L += kin * kinetic_all(s, UN);
    free(j); free(nh);
    return L;
}

/* Forward nsteps of the continuous full cycle from the current state and the reverse sweep.
 * out[0] = L, out[1] = dL/dD (1/J), out[2] = dL/dr0 (1/m), out[3] = dL/dI0 (m^2/W).
 * The context's state is left unchanged. */
void oracle_full_grad(ostate* s, int32_t nsteps, const double* cw, double kin, double* out)
{
    int nx = s->c.nx, nz = s->c.nz;
    size_t nn = (size_t)nx * (nz + 1);
    ftraj T;
    traj_alloc(s, &T, nsteps);
    double L = traj_forward(s, &T, cw, kin, s->E0);
    int N = nsteps;
    /* adjoints of the final state */
    double *lX[2] = {0, 0}, *lZ[2] = {0, 0}, *lU[2] = {0, 0};
    for (int sp = 0; sp < s->nsp; sp++) {
        size_t n = (size_t)s->np[sp];
        lX[sp] = calloc(n ? n : 1, sizeof(double));
        lZ[sp] = calloc(n ? n : 1, sizeof(double));
        lU[sp] = calloc(3 * (n ? n : 1), sizeof(double));
        double mc2w = s->w * s->m[sp] * O_C * O_C;
        const double* u = T.U[sp] + 3 * (size_t)N * n;
        for (size_t p = 0; p < n; p++) {
            double g = sqrt(1.0 + u[3 * p] * u[3 * p] + u[3 * p + 1] * u[3 * p + 1] + u[3 * p + 2] * u[3 * p + 2]);
            for (int d = 0; d < 3; d++) lU[sp][3 * p + d] = kin * mc2w * u[3 * p + d] / g;
        }
    }
    double gD = 0.0, gr0 = 0.0, gE0 = 0.0;
    double* nh = malloc(sizeof(double) * nn);
    double* lam = calloc(nn, sizeof(double));
    double* lF = calloc(6 * nn, sizeof(double));
    double* lj = calloc(3 * nn, sizeof(double));
    if (s->pair[0]) {
        double *xN = T.X[0] + (size_t)N * s->np[0], *zN = T.Z[0] + (size_t)N * s->np[0];
        dens_cont(s, xN, zN, s->np[0], nh);
        deposit_transpose(s, cw, xN, zN, s->np[0], lX[0], lZ[0]);
        for (size_t c = 0; c < nn; c++) gr0 += cw[c] * 3.0 * nh[c] / s->r0;
    }
    for (int t = N - 1; t >= 0; t--) {
        const double* F = T.F + (size_t)t * 6 * nn;
        /* Maxwell of step t: adjoint of the new fields -> of the old fields and of j */
        if (s->c.mode == 0) maxwell_cont_T(s, lF, lj, s->step + t, &gE0);
        else memset(lj, 0, sizeof(double) * 3 * nn);
        if (s->pair[0]) dens_cont(s, T.X[0] + (size_t)t * s->np[0], T.Z[0] + (size_t)t * s->np[0], s->np[0], nh);
        memset(lam, 0, sizeof(double) * nn);
        for (int sp = 0; sp < s->nsp; sp++) {
            size_t n = (size_t)s->np[sp];
            double sg = s->q[sp] > 0 ? 1.0 : (s->q[sp] < 0 ? -1.0 : 0.0);
            double q = s->q[sp], m = s->m[sp], dt = s->dt;
            double eps = q * dt / (2.0 * m * O_C), fk = dt / (2.0 * m * O_C);
            for (size_t p = 0; p < n; p++) {
                double x = T.X[sp][t * n + p], z = T.Z[sp][t * n + p];
                const double* u = T.U[sp] + 3 * (t * n + p);
                pstep P;
                particle_fwd(s, sp, F, nh, x, z, u, &P);
                /* adjoints of the new state, plus the current's dependence on it */
                double lx1 = lX[sp][p], lz1 = lZ[sp][p], luf[3];
                for (int d = 0; d < 3; d++) luf[d] = lU[sp][3 * p + d];
                double lx0 = 0.0, lz0 = 0.0;
                if (s->c.mode == 0 && sg != 0.0) {
                    double g5[5] = {0, 0, 0, 0, 0};
                    cur_cont_T(s, sg, x, z, P.x1u, P.z1, P.by, lj, lj + nn, lj + 2 * nn, g5);
                    lx0 += g5[0]; lz0 += g5[1]; lx1 += g5[2]; lz1 += g5[3];
                    /* by = ufin_y / gamma */
                    double gg = P.gfin;
                    for (int d = 0; d < 3; d++) luf[d] += g5[4] * ((d == 1 ? 1.0 / gg : 0.0) - P.ufin[1] * P.ufin[d] / (gg * gg * gg));
                }
                /* wall mirror */
                double lzn = lz1;
                if (P.refl) { lzn = -lz1; luf[2] = -luf[2]; }
                /* move: xn = x + cs uf_x, zn = z + cs uf_z, cs = c dt / (gamma dx) */
                double udl = (P.uf[0] * lx1 + P.uf[2] * lzn) / (P.g * P.g);
                double lu[3];
                lu[0] = luf[0] + P.cs * (lx1 - P.uf[0] * udl);
                lu[1] = luf[1] + P.cs * (0.0 - P.uf[1] * udl);
                lu[2] = luf[2] + P.cs * (lzn - P.uf[2] * udl);
                lx0 += lx1;
                lz0 += lzn;
                /* Boris transpose: lu is the adjoint of uf = up + a */
                double la[3], lup[3], lupr[3], lsv[3], lt[3], lum[3];
                for (int d = 0; d < 3; d++) { la[d] = lu[d]; lup[d] = lu[d]; }
                /* up = um + upr x sv */
                for (int d = 0; d < 3; d++) lum[d] = lup[d];
                lupr[0] = P.sv[1] * lup[2] - P.sv[2] * lup[1];
                lupr[1] = P.sv[2] * lup[0] - P.sv[0] * lup[2];
                lupr[2] = P.sv[0] * lup[1] - P.sv[1] * lup[0];
                lsv[0] = lup[1] * P.upr[2] - lup[2] * P.upr[1];
                lsv[1] = lup[2] * P.upr[0] - lup[0] * P.upr[2];
                lsv[2] = lup[0] * P.upr[1] - lup[1] * P.upr[0];
                /* upr = um + um x t */
                lum[0] += lupr[0] + (P.t[1] * lupr[2] - P.t[2] * lupr[1]);
                lum[1] += lupr[1] + (P.t[2] * lupr[0] - P.t[0] * lupr[2]);
                lum[2] += lupr[2] + (P.t[0] * lupr[1] - P.t[1] * lupr[0]);
                lt[0] = lupr[1] * P.um[2] - lupr[2] * P.um[1];
                lt[1] = lupr[2] * P.um[0] - lupr[0] * P.um[2];
                lt[2] = lupr[0] * P.um[1] - lupr[1] * P.um[0];
                /* sv = 2 t / (1 + t.t) */
                double tl = P.t[0] * lsv[0] + P.t[1] * lsv[1] + P.t[2] * lsv[2], d1 = 1.0 + P.t2;
                for (int d = 0; d < 3; d++) lt[d] += 2.0 * lsv[d] / d1 - 4.0 * tl * P.t[d] / (d1 * d1);
                /* t = tfac B, tfac = q dt / (2 m gm) */
                double lB[3], ltf = 0.0;
                for (int d = 0; d < 3; d++) { lB[d] = P.tfac * lt[d]; ltf += P.B[d] * lt[d]; }
                double lgm = -P.tfac / P.gm * ltf;
                for (int d = 0; d < 3; d++) lum[d] += lgm * P.um[d] / P.gm;
                /* um = u + a */
                for (int d = 0; d < 3; d++) la[d] += lum[d];
                for (int d = 0; d < 3; d++) lU[sp][3 * p + d] = lum[d];
                /* a = eps E + fk Fp: field gathers */
                if (s->c.mode == 0)
                    for (int f = 0; f < 6; f++) {
                        double lv = f < 3 ? eps * la[f] : lB[f - 3];
                        gather_arr(s, F + f * nn, x, z, k_stag[f][0], k_stag[f][1], lF + f * nn, lv, &lx0, &lz0);
                    }
                if (s->pair[sp]) {
                    double lFx = fk * la[0], lFz = fk * la[2];
                    gD += (lFx * P.Fp[0] + lFz * P.Fp[2]) / s->D;
                    gr0 += lFx * (P.dxr + P.dxn * 3.0 * P.n / s->r0 + P.dxq * 3.0 * P.qx / s->r0);
                    gr0 += lFz * (P.dzr + P.dzn * 3.0 * P.n / s->r0 + P.dzq * 3.0 * P.qz / s->r0);
                    double ln = lFx * P.dxn + lFz * P.dzn, lqx = lFx * P.dxq, lqz = lFz * P.dzq;
                    lx0 += ln * P.qx + lqz * P.gxz;
                    lz0 += ln * P.qz + lqx * P.gxz;
                    int64_t i, k; double fx, fz, n_, a1, a2, a3;
                    gather_cont(s, nh, x, z, &n_, &a1, &a2, &a3, &i, &k, &fx, &fz);
                    size_t c00 = (size_t)k * nx + imod(i, nx), c10 = (size_t)k * nx + imod(i + 1, nx);
                    size_t c01 = (size_t)(k + 1) * nx + imod(i, nx), c11 = (size_t)(k + 1) * nx + imod(i + 1, nx);
                    lam[c00] += ln * (1 - fx) * (1 - fz) - lqx * (1 - fz) - lqz * (1 - fx);
                    lam[c10] += ln * fx * (1 - fz) + lqx * (1 - fz) - lqz * fx;
                    lam[c01] += ln * (1 - fx) * fz - lqx * fz + lqz * (1 - fx);
                    lam[c11] += ln * fx * fz + lqx * fz + lqz * fx;
                }
                lX[sp][p] = lx0;
                lZ[sp][p] = lz0;
            }
        }
        if (s->pair[0]) deposit_transpose(s, lam, T.X[0] + (size_t)t * s->np[0], T.Z[0] + (size_t)t * s->np[0],
                                          s->np[0], lX[0], lZ[0]);
    }
    out[0] = L;
    out[1] = gD;
    out[2] = gr0;
    out[3] = s->c.I0 > 0 ? gE0 * s->E0 / (2.0 * s->c.I0) : 0.0;
    for (int sp = 0; sp < s->nsp; sp++) { free(lX[sp]); free(lZ[sp]); free(lU[sp]); }
    free(nh); free(lam); free(lF); free(lj);
    traj_free(&T);
}

/* Loss of the continuous full cycle after nsteps with D, r0, I0 overriding the configuration
 * (for finite differences); the context's state is left unchanged. */
double oracle_full_loss(ostate* s, int32_t nsteps, const double* cw, double kin, double D_J, double r0_m, double I0)
{
    double Dsave = s->D, r0save = s->r0;
    s->D = D_J;
    s->r0 = r0_m;
    ftraj T;
    traj_alloc(s, &T, nsteps);
    double L = traj_forward(s, &T, cw, kin, sqrt(2.0 * I0 / (O_EPS0 * O_C)));
    traj_free(&T);
    s->D = Dsave;
    s->r0 = r0save;
    return L;
}

double oracle_E0(const ostate* s) { return s->E0; }
