// Internal types and launch declarations of the GB300 PIC library (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace gbpic {

// CODATA 2018
constexpr double kC = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKb = 1.380649e-23;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kPi = 3.14159265358979323846;

constexpr int kQBits = 16;           // fixed-point bits per cell along one axis
constexpr int32_t kQOne = 1 << kQBits;

// status word bits (device, sticky)
constexpr unsigned kErrNan = 1u;
constexpr unsigned kErrMove = 2u;
constexpr unsigned kErrOverflow = 8u;    // more particles per cell than the int64 node sums are proven for

typedef unsigned long long u64;

// One species in structure-of-arrays form. Two buffers: `a` is the live one, `b` the target of
// the cell sort (swapped after each sort).
struct SpeciesBuf {
    int32_t* cell;
    float* fx;
    float* fy;           // 3D only (NULL in 2D)
    float* fz;
    float* ux;
    float* uy;
    float* uz;
};

struct Species {
    SpeciesBuf a, b;
    int32_t* tile_start;   // ntiles + 1 offsets into `a` (from the last sort)
    int64_t n, cap;
    int32_t ppc;
    float e_kick;          // q dt / (2 m c)          per V/m
    float b_rot;           // q dt / (2 m)            per T (divided by gamma)
    float p_kick;          // dt (D / r0) / (2 m c)    per unit dimensionless pair force
    int32_t jsign;         // charge sign for the current (0: neutral)
    int32_t pair;          // carries the pair force and the node density
    double mass, uth;
};

// The embedded-atom form (pot_mode 3), energies in units of D, r in units of r0: f(r) =
// exp(-beta (r - 1)), phi(r) = phi exp(-gamma (r - 1)), F(rho) = -ec (1 - (alpha/beta) ln x)
// x^(alpha/beta) - 3 phi x^(gamma/beta), x = rho / 6.
struct EamP {
    float ec, phi, alpha, beta, gamma;
};
inline EamP eam_params(const pic_config& cfg)
{
    EamP e;
    e.ec = (float)(cfg.eam_ec / cfg.D_eV);
    e.phi = (float)(cfg.eam_phi / cfg.D_eV);
    e.alpha = (float)cfg.eam_alpha;
    e.beta = (float)cfg.eam_beta;
    e.gamma = (float)cfg.eam_gamma;
    return e;
}

// pot_mode 3 asks for the cubic lattice and positive parameters (eam_phi may be 0).
inline bool eam_config_ok(const pic_config& cfg)
{
    if (cfg.pot_mode != 3) return true;
    return cfg.lattice == PIC_LATTICE_CUBIC && cfg.eam_ec > 0 && cfg.eam_ec < 1e3 && cfg.eam_phi >= 0 &&
           cfg.eam_phi < 1e3 && cfg.eam_alpha > 0 && cfg.eam_alpha < 1e3 && cfg.eam_beta > 0 && cfg.eam_beta < 1e3 &&
           cfg.eam_gamma > 0 && cfg.eam_gamma < 1e3;
}

// The second parameter of the device pair functions: the Morse stiffness for pot_mode 2, the
// attractive factor of the altered potential otherwise (the functions take it as c_att).
inline float pot_param(const pic_config& cfg) { return (float)(cfg.pot_mode == 2 ? cfg.morse_a : cfg.c_att); }

// The potential code the device pair functions and the particle-kernel instances take: pot_mode
// in bits 0-1, the HCP lattice in bit 2 (kLatHcp).
inline int pot_code(const pic_config& cfg) { return cfg.pot_mode | (cfg.lattice == PIC_LATTICE_HCP ? 4 : 0); }

// Everything a kernel of the step needs, passed by value.
struct StepArgs {
    int32_t nx, nz, T, ntx, ntz, ntiles, W;   // W: window edge (nodes) of a tile
    unsigned nx_magic;                        // floor(2^32 / nx) for the cell -> (i, k) split
    int32_t full;                             // fields and Lorentz force on
    float cdt_dx;                             // c dt / dx
    float rho_s;                              // node sum -> n / n0
    float h_coef;                             // r0 / (6 dx): h = -h_coef * dn * n^(-4/3)
    int32_t pot_mode;
    float c_att, s_rep;
    const float* F[6];
    const u64* rho_cur;
    u64* rho_next;
    u64* J[3];
    unsigned* status;
    int32_t nsp;
    Species sp[2];
    EamP eam;                                 // the embedded-atom form's parameters (pot_mode 3)
    float jy_scale;                           // 2^jy_bits: the J_y code V = rint(beta_y 2^jy_bits)
    float jy_zero;                            // 2^-(jy_bits + 1): |u_y| below it gives V = 0
};

struct Ctx {
    pic_config cfg;
    cudaStream_t stream;
    int device;
    int nsm;
    // derived
    double dt, w, r0, D, rho_scale, E0, omega, t_ant;
    int32_t dims, ny, nty;  // 2 or 3; cells and tiles along y (1 in 2D)
    int32_t nx, nz, T, ntx, ntz, ntiles, W, k_ant;
    size_t nn;            // (nz + 1) * nx
    int32_t nkeys;        // ntiles * T * T
    int32_t nsp;
    Species sp[2];
    // grids
    float* F[6];
    u64* J[3];
    u64* rho[2];
    int32_t cur;          // rho[cur] holds the node density at the current positions
    float* mur_save;      // 8 * nx
    float* ant_c;         // nx: amplitude * cos(phase(x)) at x = i + 1/2
    float* ant_s;         // nx: amplitude * sin(phase(x))
    float* ant;           // 2: antenna scalars of the current step (written on the device)
    // scratch
    int32_t* keys_count;  // nkeys + 1
    int32_t* keys_off;    // nkeys + 1
    int32_t* scan_tmp;    // block sums
    double* partials;     // energy block partials
    double* red_out;      // 8 doubles
    unsigned* status;     // 8 words: sticky error bits, validation count, particle-kernel ticket, spare,
                          // largest particle count of one block of 4^dims cells per species (last sort)
    int32_t jy_bits;      // resolution of the J_y code (2D full mode)
    int32_t count_limit;  // particles per block of 4^dims cells (both species) for which no int64
                          // node sum can overflow
    int64_t step;
    int32_t steps_since_sort;
    int sticky;
    int in_batch;         // stepped by a batch (pic_step refuses)
    // timing
    int timing;
    cudaEvent_t ev[4];
    double ms[3];
    int64_t nlaunch[4];
};

// Laser antenna of one simulation (scalars evaluated on the device each step).
struct AntennaParams {
    int on;
    double dt, t_ant, tau_fwhm, omega, coef;
};

// Everything a field kernel needs for one simulation.
struct FieldArgs {
    int nx, nz, k_ant;
    float h_b;           // dt / (2 dx)      (half step of B)
    float h_e;           // c^2 dt / dx      (full step of E)
    float cj;            // J2x, J2z -> dt J / eps0
    float cjy;           // J6y -> dt J_y / eps0
    float mur;           // (c dt - dx) / (c dt + dx)
    float* F[6];
    const u64* J[3];
    float* save;         // 8 * nx: Ex(0) Ex(1) Ex(nz-1) Ex(nz) Ey(0) Ey(1) Ey(nz-1) Ey(nz) before the E step
    const float* antc;   // nx: amplitude * cos(phase(x))
    const float* ants;   // nx: amplitude * sin(phase(x))
    const float* ant;    // 2: this step's antenna scalars
    int k_flux;          // node row below the antenna: Poynting flux of the injected energy
    double* flux;        // accumulates sum (Ex By - Ey Bx) over that row at the half step
};

// kernels launched from the host side of the library (defined in the .cu files)
void launch_init_particles(Ctx& c, int s, cudaStream_t st);
void launch_sort_species(Ctx& c, int s, cudaStream_t st, int64_t* launches);
// Fixed-point range: the J_y code resolution for a 2D full-mode slab of n particles per cell (both
// species) and the particle count per block of 4^dims cells up to which every int64 node sum is
// proven exact.
int choose_jy_bits(int64_t n_per_cell);
int64_t count_limit(int dims, int full, int jy_bits);
void launch_deposit_density(Ctx& c, u64* out, cudaStream_t st);
void launch_crater_profile(Ctx& c, const u64* rho0, double depth_scale, double* out, cudaStream_t st);
// One device-to-device copy (src != NULL) or clear (src == NULL) of `bytes` bytes.
struct CopySeg {
    const void* src;
    void* dst;
    size_t bytes;
};
constexpr int kMaxCopySegs = 32;
constexpr int kMaxDevices = 64;   // per-device launch attributes are tracked up to this device index
// copies / clears a list of segments with a vectorised kernel (one launch per 32 segments); returns
// the number of launches
int launch_copy_segments(const Ctx& c, const CopySeg* segs, int n, cudaStream_t st);
void launch_cell_temperature(Ctx& c, int s, double* work, double* T, cudaStream_t st);
void launch_set_temperature(Ctx& c, int s, const double* T, double T_from, cudaStream_t st);
void launch_pair_force_probe(Ctx& c, int64_t n, const int32_t* cell, const float* fx, const float* fz, int pot_mode,
                             double c_att, double s_rep, float* out, cudaStream_t st);
void launch_pair_force(Ctx& c, float* out, cudaStream_t st);
void launch_validate(Ctx& c, const SpeciesBuf& b, int64_t n, unsigned* bad, cudaStream_t st);
void launch_particle_step(Ctx& c, const StepArgs& a, cudaStream_t st);
void launch_fields(Ctx& c, cudaStream_t st, int64_t step, int64_t* launches);
// the field arguments of every slab of a batch, passed in the kernels' parameter block
constexpr int kMaxFieldSlabs = 48;
struct FieldBatch {
    FieldArgs f[kMaxFieldSlabs];
    int rb[kMaxFieldSlabs + 1];      // first (row, 256-node segment) block of each slab
    int n;
};
void launch_fields_batch(const FieldBatch& P, const AntennaParams* ap_dev, long long* step_dev, float* ant_dev,
                         cudaStream_t st);
void field_row_blocks(FieldBatch& P);
FieldArgs make_field_args(const Ctx& c);
AntennaParams make_antenna_params(const Ctx& c);
void launch_particle_step_batch(const StepArgs* args_dev, const int* tile_base_dev, int nslab, int total_tiles,
                                int full, int pot, int maxW, int nsm, cudaStream_t st);
size_t particle_smem_bytes(int W);
void launch_particle_step3(Ctx& c, cudaStream_t st);
void launch_deposit_density3(Ctx& c, u64* out, cudaStream_t st);
void launch_pair_force3(Ctx& c, float* out, cudaStream_t st);
void launch_fields3(Ctx& c, cudaStream_t st, int64_t step, int64_t* launches);
void launch_energy3(Ctx& c, cudaStream_t st, double* host_out5);
void launch_init_particles3(Ctx& c, int s, cudaStream_t st);
void launch_adjoint_seed(Ctx& c, double kin, const double* w_nodes, float* lam_pos, float* lam_u, float* lam_nodes,
                         double* r0_out, cudaStream_t st);
void launch_adjoint_step(Ctx& c, float* lam_pos, float* lam_u, float* lam_nodes, double* grads, cudaStream_t st);
void launch_node_functional(Ctx& c, const double* w_nodes, double* dev_out, cudaStream_t st);
void launch_adjoint_seed_full(Ctx& c, double kin, const double* w_nodes, float* const* lam_pos, float* const* lam_u,
                              float* lam_nodes, double* lF, float* lj, double* r0_out, cudaStream_t st);
void launch_adjoint_step_full(Ctx& c, float* const* lam_pos, float* const* lam_u, float* lam_nodes, double* lF,
                              float* lj, double* grads, cudaStream_t st);
int tile_window(int T);
void launch_energy(Ctx& c, cudaStream_t st, double* host_out5);
StepArgs make_step_args(Ctx& c);

}  // namespace gbpic

// The C ABI's opaque context (include/pic.h).
struct pic_ctx {
    gbpic::Ctx c;
    std::vector<cudaEvent_t> evpool;
    std::vector<int> evkind;    // 0 particle, 1 fields, 2 sort (pairs of events)
};
