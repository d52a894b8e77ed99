/*
 * pic.h -- C ABI of the GB300 particle-in-cell cycle with the pair-potential force of
 * Mitchell, Schumacher & Chowdhury, "Modeling crater formation in femtosecond-pulse laser
 * damage from basic principles" (arXiv:1502.07722).
 *
 * One simulation = one context (pic_ctx) on the current CUDA device. The library computes every
 * step of the cycle in its own CUDA kernels (sm_103a). It never allocates device memory: the
 * caller hands it one device workspace of pic_workspace_size() bytes (the Python binding takes
 * it from PyTorch's allocator) and a CUDA stream. All work is queued on that stream.
 *
 * Geometry (paper: 2D simulation with three-component vectors, positions in-plane):
 *   cells (i, k), i = 0..nx-1 along x (periodic), k = 0..nz-1 along z (walls at z = 0, nz).
 *   Node rows k = 0..nz; grids are (nz+1) x nx, row-major (index k*nx + i), even for the
 *   half-row components (their row nz is unused).
 *   Yee positions: Ex (i+1/2,k)  Ey (i,k)  Ez (i,k+1/2)  Bx (i,k+1/2)  By (i+1/2,k+1/2)  Bz (i+1/2,k).
 *   A particle is (cell = k*nx + i, fx, fz in [0,1), ux, uy, uz = gamma v / c), FP32.
 *   Species 0: Cu ions (or neutral atoms in the transport mode) -- the pair-potential species.
 *   Species 1: electrons (full mode only).
 *
 * Fixed point: a coordinate x (cells) deposits with X = i*2^16 + rint(f * 2^16); node weight
 * S_j = max(0, 2^16 - |X - 2^16 j|). Node sums are int64 and exact, so they are identical for
 * any summation order (deterministic) and bit-comparable with a CPU reference. The out-of-plane
 * current uses the code V = rint(beta_y 2^b), b = 18 unless the slab's particles per cell (both
 * species, with a quarter headroom) could overflow J6y at that resolution, then the largest b
 * that cannot. A node collects from the particles of 4 x 4 cells (4^3 in 3D); the largest
 * contribution of one particle is 6 * 2^(32+b) to J6y, 2^34 to J2x/J2z and 2^33 to the density
 * in 2D, 3 * 2^44 to a 3D current and 2^43 to the 3D density. So the sums are exact while no cell
 * holds more than 2^63 / (16 * 6 * 2^(32+b)) particles (85 at b = 18) in the 2D full mode, 2730
 * in the 3D full mode, 2^28 and 2^17 without currents (transport mode). pic_init refuses a slab
 * whose initial particles per cell exceed the limit (PIC_EOVERFLOW); every cell sort checks the
 * largest cell count of each species and raises a sticky PIC_EOVERFLOW when their sum exceeds it
 * (a pile-up between two sorts is found at the next sort).
 *
 * Return codes: 0 on success, a negative PIC_E* code on error. Errors raised inside kernels
 * (non-finite momentum, a move of a cell or more, a cell holding more particles than the fixed-point
 * range allows) are sticky: pic_step reports them and every later call on the context returns them
 * until pic_free.
 */
#ifndef GBPIC_PIC_H
#define GBPIC_PIC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PIC_OK = 0,
    PIC_EINVAL = -1,     /* bad argument or configuration                                  */
    PIC_ENOMEM = -2,     /* workspace too small / particle count above capacity            */
    PIC_ECUDA = -3,      /* a CUDA runtime call failed                                     */
    PIC_ENAN = -4,       /* a particle momentum became non-finite                          */
    PIC_EMOVE = -5,      /* a particle moved a cell or more in one step (CFL is violated)  */
    PIC_ESTATE = -6,     /* call not valid in this mode (e.g. fields in transport mode)    */
    PIC_EOVERFLOW = -7   /* more particles in one cell than the int64 node sums are proven
                            exact for: refused at init, sticky when a sort finds a pile-up    */
};

enum { PIC_MODE_FULL = 0, PIC_MODE_TRANSPORT = 1 };
enum { PIC_LASER_NONE = 0, PIC_LASER_PLANE = 1, PIC_LASER_GAUSSIAN = 2 };
enum { PIC_EX = 0, PIC_EY = 1, PIC_EZ = 2, PIC_BX = 3, PIC_BY = 4, PIC_BZ = 5 };

/* Physical inputs. Derived quantities (dt, weights, E0, ...) are computed by pic_init. */
typedef struct pic_config {
    int32_t nx, nz;          /* cells along x (periodic) and z (walls); 3 <= n < 32768          */
    int32_t slab_k;          /* the slab fills cell rows k < slab_k at init                     */
    int32_t mode;            /* PIC_MODE_FULL: Cu+ ions, electrons, fields (ion_charge = 1);
                                PIC_MODE_TRANSPORT: neutral atoms and the pair force only        */
    int32_t ppc_ion, ppc_electron;   /* macroparticles per slab cell (equal in the full mode)   */
    int32_t pot_mode;        /* 0: Eq. (3) as printed; 1: altered L-J (s_rep below r0, c_att above);
                                2: Morse, U = D [e^(-2a(r/r0-1)) - 2 e^(-a(r/r0-1))], a = morse_a (the
                                paper: the density-to-distance mapping takes any pair potential,
                                the Morse potential among them); its minimum is -D at r0 like Eq. (3);
                                3: the embedded-atom form (eam_* below)                            */
    int32_t laser_profile;   /* PIC_LASER_*                                                     */
    int32_t tile;            /* tile edge in cells for particle binning (0: 16 in 2D, 10 in 3D)  */
    int32_t sort_every;      /* steps between cell sorts (0: only after init / set_particles)  */
    int64_t max_particles;   /* per-species capacity (0: the initial count)                    */
    double dx;               /* cell size (m), square cells                                     */
    double cfl;              /* dt = cfl * dx / (c sqrt 2) unless dt_override > 0               */
    double dt_override;      /* s                                                               */
    double n_atoms;          /* solid density (m^-3), paper: 8.5e22 cm^-3 for copper            */
    double T_ion_K, T_electron_eV;   /* Maxwellian start                                        */
    double ion_charge;       /* e units: 1 (full mode) or 0 (transport mode)                    */
    double ion_mass_amu;
    double D_eV;             /* Eq. (3) dissociation energy                                     */
    double r0;               /* Eq. (3) equilibrium distance (m); <= 0: n_atoms^(-1/3)          */
    double c_att, s_rep;     /* altered-potential factors (pot_mode 1)                          */
    double lambda, I0, tau_fwhm, w0, t_peak;  /* laser: m, W/m^2, s (intensity FWHM), m, s:
                                the pulse peak reaches the slab surface z = slab_k at t_peak    */
    uint64_t seed;           /* initial-state generator seed                                    */
    int32_t ny;              /* cells along y (periodic), 3D only                               */
    int32_t dims;            /* 2 (default when 0) or 3. In 3D: grids (nz+1) x ny x nx, index
                                (k*ny + j)*nx + i; a particle also has fy; fixed point 2^14 per
                                axis (weights of a node sum in units 2^-42); current J6x, J6y, J6z
                                with J_x = J6x * e w / (6 * 2^42 dx^2 dt); dt = cfl dx / (c sqrt 3) */
    int32_t temp_profile;    /* PIC_TEMP_UNIFORM: species 0 starts at T_ion_K everywhere.
                                PIC_TEMP_SPOT: the lattice temperature a laser spot left
                                behind (paper, Fig. 2 and the initialisation paragraph: the atomic-
                                transport run starts from the lattice temperature after electrons
                                and lattice equilibrate), for species 0 at its initial position
                                (x, z) in cells: T = T_ion_K + (T_spot_K - T_ion_K)
                                * exp(-2 ((x - nx/2) dx / spot_w)^2) * exp(-(slab_k - z) dx / spot_depth);
                                in 3D the lateral term takes the radius from the axis,
                                ((x - nx/2)^2 + (y - ny/2)^2) dx^2 / spot_w^2 */
    int32_t lattice;         /* PIC_LATTICE_CUBIC (0): the paper's cubic lattice, six neighbours on the
                                axes. PIC_LATTICE_HCP (1): hexagonal close-packed (the paper: the method
                                adapts to it), ideal axial ratio, c axis along z: six basal neighbours,
                                three above and three below the basal plane, both sublattices' out-of-
                                plane triples averaged (weight 1/2 each). Eq. (2) along each neighbour
                                direction e puts it at rbar / (1 - (grad rbar . e) / 2); the force is the
                                sum of U'(r_e) e. r0 stays the equilibrium nearest-neighbour distance. */
    double T_spot_K;         /* peak temperature on the axis at the surface (K)                  */
    double spot_w;           /* 1/e^2 radius of the lateral Gaussian (m)                          */
    double spot_depth;       /* 1/e depth of the temperature below the surface (m)                */
    double morse_a;          /* Morse stiffness alpha r0 (dimensionless, 0 < morse_a < 1000) for
                                pot_mode 2; unused otherwise                                      */
    double eam_ec, eam_phi;  /* pot_mode 3, the embedded-atom form on the cubic lattice (the paper:
                                other potentials adapt to its density mapping), r in units of r0:
                                f(r) = exp(-eam_beta (r - 1)) per neighbour, pair term
                                phi(r) = eam_phi exp(-eam_gamma (r - 1)), embedding energy
                                F(rho) = -eam_ec (1 - (a/b) ln x) x^(a/b) - 3 eam_phi x^(g/b),
                                x = rho / 6 (a, b, g = eam_alpha, eam_beta, eam_gamma), so that a
                                uniform lattice follows -eam_ec (1 + a(r - 1)) e^(-a(r - 1)). Atom i's
                                embedding density sums f over its six Eq. (2) neighbours; neighbour j's
                                is 6 f(n_j^(-1/3)), n_j the density at j's position (n + s dn along the
                                axis, s its offset); each bond pulls with phi' + (F'(rho_i) + F'(rho_j)) f'.
                                eam_ec, eam_phi in eV (> 0); exponents > 0. Cubic lattice only.       */
    double eam_alpha, eam_beta, eam_gamma;
} pic_config;

#define PIC_TEMP_UNIFORM 0
#define PIC_TEMP_SPOT 1
#define PIC_LATTICE_CUBIC 0
#define PIC_LATTICE_HCP 1

typedef struct pic_info {
    double dt;               /* s                                                               */
    double weight;           /* real atoms (or electrons) per macroparticle, per metre of y     */
    double rho_scale;        /* pair node sum -> density in units of n0 = r0^-3                  */
    double r0;               /* m                                                               */
    double time;             /* s, simulated time of the current state                          */
    int64_t step;
    int64_t num_particles[2];
    int32_t nspecies;
    int32_t ntiles;
} pic_info;

/* Energies in J per metre of y. Kinetic energies use the stored (half-step) momenta; field
 * energy weights the wall node rows by 1/2; pair energy is, per atom, half the sum of U over its
 * six cubic-lattice neighbours (+-x, +-z from Eq. 2, +-y at rbar). */
typedef struct pic_energy_t {
    double kinetic_ion, kinetic_electron, field_E, field_B, pair;
    int64_t step;
    double injected;   /* energy the laser sent towards the slab so far: the Poynting flux through
                          the node row (plane) below the antenna, summed over the steps */
} pic_energy_t;

typedef struct pic_ctx pic_ctx;

/* sizeof(pic_config) as this library was built: a binding checks its own copy of the struct
 * against it. Host only; no errors. (Not a step of the paper's method.) */
PIC_API size_t pic_config_bytes(void);

/* Bytes of device workspace pic_init needs for cfg. Returns PIC_EINVAL for an invalid cfg and
 * PIC_EOVERFLOW for a slab whose particles per cell exceed the fixed-point range (see above);
 * makes no CUDA call. */
PIC_API int pic_workspace_size(const pic_config* cfg, size_t* bytes);

/* Create a simulation on the current device: generate the initial slab (paper: the damage
 * simulation is initialised for target density and temperature), sort it into tiles and
 * deposit the initial node density. workspace: device pointer, 256-byte aligned, owned by the
 * caller and kept alive until pic_free. stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out receives the context (host memory owned by the library). */
PIC_API int pic_init(const pic_config* cfg, void* workspace, size_t workspace_bytes, void* stream, pic_ctx** out);

/* Release the host-side context. The workspace stays the caller's. NULL is accepted. */
PIC_API void pic_free(pic_ctx* ctx);

/* Advance nsteps PIC cycles (paper: the PIC cycle is evaluated for each time step):
 * node density -> pair force (Eqs. 1-3) -> Lorentz + pair push -> current deposition ->
 * node density at the new positions -> Maxwell (Yee) update. Synchronises the stream at the end
 * to read the sticky status word; returns it. */
PIC_API int pic_step(pic_ctx* ctx, int32_t nsteps);

/* Node density of the pair species at the current positions (paper: weights interpolated to
 * the nearest surrounding nodes give the node density): dev_out receives (nz+1)*nx int64 sums
 * in units 2^-32 of one macroparticle (device pointer, caller-owned). *scale_out (host, may be
 * NULL) receives the factor from a sum to a density in m^-3. Recomputed from the particles. */
PIC_API int pic_deposit_density(pic_ctx* ctx, int64_t* dev_out, double* scale_out);

/* Crater profile (paper: after the crater has solidified its width and depth are measured from
 * the density map; Eq. 5 turns the width into a threshold fluence). For every column of nodes
 * (nx in 2D, ny*nx in 3D, index j*nx + i) the material missing from the original slab as a
 * thickness of solid-density material, in metres:
 *     dev_out[col] = dx * scale / n_atoms * sum_{k = 0..slab_k} (dev_rho0 - rho)(k, col),
 * rho the node sums of the pair species at the current positions, dev_rho0 earlier node sums in
 * the layout of pic_deposit_density (typically taken right after pic_init), scale the factor
 * pic_deposit_density returns. The column sums are exact integers. Device pointers, caller-owned;
 * asynchronous on the context's stream. Errors: PIC_EINVAL for NULL pointers. */
PIC_API int pic_crater_profile(pic_ctx* ctx, const int64_t* dev_rho0, double* dev_out);

/* Lattice temperature per cell of one species (paper: the transport run starts from the lattice
 * temperature the laser-interaction run leaves once electrons and lattice have equilibrated):
 * for the N particles of `species` in a cell, T = m c^2 / (3 k_B) * sum |u - mean u|^2 / (N - 1)
 * in K (u = gamma v / c; the spread about the cell's mean flow); cells with fewer than two
 * particles get 0. dev_T: double[ncell], ncell = nz*nx (2D, index k*nx + i) or nz*ny*nx (3D,
 * (k*ny + j)*nx + i); dev_work: caller-owned scratch of 5*ncell doubles. FP64 per-cell sums by
 * atomics (the last bits depend on their order). Asynchronous on the context's stream.
 * Errors: PIC_EINVAL (NULL pointers, species not present). */
PIC_API int pic_cell_temperature(pic_ctx* ctx, int32_t species, double* dev_work, double* dev_T);

/* Re-temper one species to a temperature map: momenta drawn at the uniform temperature T_from (K)
 * become the same draws at the temperature of their cell, u -> u sqrt(T_cell / T_from), taken in
 * FP64 and rounded to FP32 (the two-stage coupling: a transport context started at T_from takes
 * the lattice temperature of a laser-stage context). dev_T: double[ncell] as for
 * pic_cell_temperature, every value >= 0. Asynchronous on the context's stream.
 * Errors: PIC_EINVAL (NULL pointer, species not present, T_from <= 0). */
PIC_API int pic_set_temperature(pic_ctx* ctx, int32_t species, const double* dev_T, double T_from);

/* Conservative remap of a cell-centred field (a lattice-temperature map) between two grids of
 * square cells, for the two-stage coupling when the stages use different cells (paper: the
 * laser-interaction run, on much finer cells than the transport run, hands its lattice
 * temperature to the transport run). The grids are placed on each other by the slab's surface
 * and the laser axis: cell (i, j, k) of a grid (nx, ny, nz, dx, surface) spans
 * x in [(i - nx/2) dx, (i + 1 - nx/2) dx], y likewise with ny (3D), and depth coordinate
 * [(k - surface) dx, (k + 1 - surface) dx], surface being the first row of cells above the slab
 * (slab_k). Each destination cell takes the volume-weighted mean of the source cells it
 * overlaps; the part of it outside the source grid counts as `fill` (the source grid's periodic
 * x is not continued: its lateral edge is the edge of the laser stage's data). dims: 2 (ny
 * ignored, index k*nx + i) or 3 (index (k*ny + j)*nx + i). dev_src: double[src cells],
 * dev_dst: double[dst cells], device pointers, caller-owned, not overlapping. FP64 throughout;
 * asynchronous on `stream` (a cudaStream_t, NULL for the default stream); allocates nothing.
 * Errors: PIC_EINVAL (NULL pointers, dims not 2 or 3, an extent below 1, dx <= 0, a surface
 * outside 0..nz), PIC_ECUDA (launch failure). */
PIC_API int pic_regrid_cells(int32_t dims, const double* dev_src, int32_t src_nx, int32_t src_ny, int32_t src_nz,
                             double src_dx, int32_t src_surface, double* dev_dst, int32_t dst_nx, int32_t dst_ny,
                             int32_t dst_nz, double dst_dx, int32_t dst_surface, double fill, void* stream);

/* Pair-potential force (N, per atom) on every macro-ion from the current node density
 * (paper: Eqs. 1-3, density and gradient interpolated back to the particle). dev_out:
 * device float[3 * num_particles(0)], (Fx, Fy, Fz) per particle, in the context's particle order. */
PIC_API int pic_pair_force(pic_ctx* ctx, float* dev_out);

/* Pair-potential force (N, per atom) at n probe positions from the current node density, the
 * probes adding nothing to it (paper: the attractive correction factor is found by integrating the
 * force on a single atom leaving the target out to infinity). dev_cell, dev_fx, dev_fz: device
 * arrays of n probes (cell k*nx + i, offsets in [0,1) x [0,1]); pot_mode, c_att, s_rep as in
 * pic_config, applied to this call only (so one context yields the attractive and the repulsive
 * parts of the force separately); pot_mode 2 takes the context's morse_a and ignores c_att, s_rep;
 * the context's lattice applies. dev_out: device float[3n], (Fx, 0, Fz). A probe outside the
 * grid gets NaN. 2D contexts; asynchronous on the context's stream. Errors: PIC_EINVAL (n < 0,
 * NULL pointers with n > 0, pot_mode not 0, 1 or 2, pot_mode 2 with morse_a <= 0), PIC_ESTATE in
 * 3D. */
PIC_API int pic_pair_force_at(pic_ctx* ctx, int64_t n, const int32_t* dev_cell, const float* dev_fx,
                              const float* dev_fz, int32_t pot_mode, double c_att, double s_rep, float* dev_out);

/* Total energies of the current state, FP64 reductions on the device (paper: the pair-potential
 * cycle is energy conserving). Synchronises. host_out: host pointer. */
PIC_API int pic_energy(pic_ctx* ctx, pic_energy_t* host_out);

/* Scalars of the context. host_out: host pointer. */
PIC_API int pic_get_info(pic_ctx* ctx, pic_info* host_out);

/* Copy particles of one species out of / into the context, in the context's order. Pointers are
 * host memory when on_host != 0 (the call then synchronises), device memory otherwise. fy is the
 * y offset in 3D and is ignored (may be NULL) in 2D.
 * pic_set_particles replaces the species (n <= capacity), re-sorts it into tiles (which
 * permutes it: read it back with pic_get_particles) and re-deposits the node density. */
PIC_API int pic_get_particles(pic_ctx* ctx, int32_t species, int32_t* cell, float* fx, float* fy, float* fz,
                      float* ux, float* uy, float* uz, int32_t on_host);
PIC_API int pic_set_particles(pic_ctx* ctx, int32_t species, int64_t n, const int32_t* cell, const float* fx,
                      const float* fy, const float* fz, const float* ux, const float* uy, const float* uz,
                      int32_t on_host);

/* One field component (PIC_EX..PIC_BZ), (nz+1)*nx FP32. */
PIC_API int pic_get_field(pic_ctx* ctx, int32_t which, float* out, int32_t on_host);
PIC_API int pic_set_field(pic_ctx* ctx, int32_t which, const float* in, int32_t on_host);

/* Current of the last step, int64 fixed point, 3 planes of (nz+1)*nx: J2x at (i+1/2,k),
 * J6y at (i,k), J2z at (i,k+1/2). J_x = J2x * e w / (2^33 dx dt) A/m^2 (per unit charge sign),
 * J_y = J6y * e w c / (6 * 2^50 dx^2). */
PIC_API int pic_get_current(pic_ctx* ctx, int64_t* out3, int32_t on_host);

/* The node density the next step reads (pair species at the current positions). */
PIC_API int pic_get_density(pic_ctx* ctx, int64_t* out, int32_t on_host);

/* Sort both species by cell into tiles now (permutes the particle order). */
PIC_API int pic_sort(pic_ctx* ctx);

/* Per-kernel timing with CUDA events on the context stream. enable != 0 starts recording;
 * pic_get_timing returns the summed milliseconds and launch counts since enabling:
 * ms[0], n[0]: particle kernel; ms[1], n[1]: field kernels; ms[2], n[2]: sorts;
 * n[3]: all kernels launched by pic_step. */
PIC_API int pic_set_timing(pic_ctx* ctx, int32_t enable);
PIC_API int pic_get_timing(pic_ctx* ctx, double ms[3], int64_t n[4]);

/* ---- batched intensity sweep --------------------------------------------------------------
 * Several independent slabs (sizes, particle counts, intensities and seeds may differ; all in the
 * same mode, and either all or none with the Morse potential) advanced together: per step one persistent particle-kernel launch over the tiles of
 * every slab and one launch per field kernel for all slabs, recorded once as a CUDA graph and
 * replayed. Each slab is an ordinary context (pic_batch_slab) for reading and writing state,
 * energies and forces; pic_step on such a context returns PIC_ESTATE (step the batch instead).
 * The cell sort runs every cfgs[0].sort_every steps for all slabs. The slabs' kernel arguments
 * are copied into one constant-memory table in front of each step: two batches stepping at the
 * same time (on different streams) race on it. */
typedef struct pic_batch pic_batch;

/* Device workspace bytes for nslabs (1..48) configurations. */
PIC_API int pic_batch_workspace_size(const pic_config* cfgs, int32_t nslabs, size_t* bytes);

/* Create the batch on the current device. cfgs: host array of nslabs configurations.
 * workspace: caller-owned device memory, 256-byte aligned, kept alive until pic_batch_free.
 * stream: a non-default cudaStream_t (required: the step is recorded as a CUDA graph). */
PIC_API int pic_batch_init(const pic_config* cfgs, int32_t nslabs, void* workspace, size_t workspace_bytes,
                           void* stream, pic_batch** out);

/* Advance every slab by nsteps cycles (graph replays). Synchronises at the end and returns the
 * first slab's sticky error, if any. */
PIC_API int pic_batch_step(pic_batch* b, int32_t nsteps);

/* Context of slab i (owned by the batch; do not pic_free it). */
PIC_API int pic_batch_slab(pic_batch* b, int32_t i, pic_ctx** out);

/* With timing enabled, steps run as direct launches with CUDA events around the particle kernel
 * (ms[0]) and the field kernels (ms[1]); sorts in ms[2]. n: launches (as pic_get_timing). */
PIC_API int pic_batch_set_timing(pic_batch* b, int32_t enable);
PIC_API int pic_batch_get_timing(pic_batch* b, double ms[3], int64_t n[4]);

/* Release the batch and its slab contexts (the workspace stays the caller's). NULL is accepted. */
PIC_API void pic_batch_free(pic_batch* b);

/* Plain device arrays of one state, for pic_energy_noalloc. Species 1 is ignored in the
 * transport mode. All six field components (zeros in the transport mode) and the node density
 * of the pair species at the current positions are required. */
typedef struct pic_state_view {
    int64_t n[2];
    const int32_t* cell[2];
    const float* fx[2];
    const float* fz[2];
    const float* ux[2];
    const float* uy[2];
    const float* uz[2];
    const float* F[6];          /* (nz+1)*nx each, PIC_EX..PIC_BZ */
    const int64_t* rho;         /* (nz+1)*nx node sums, as pic_get_density returns them */
} pic_state_view;

/* The energies of pic_energy for a state given as plain device arrays, with no workspace and no
 * allocation of any kind. The paper has no counterpart: this entry point serves callers that
 * cannot allocate device memory (a host that owns every buffer and forbids further cudaMalloc,
 * or code running while another component records a CUDA graph). The reduction's scratch is a
 * fixed 40 KB array inside the library (1024 block records), reserved on every GPU that loads the
 * library until the process exits; each call writes all of it that it reads, so nothing needs
 * clearing. The first call on a device looks up the array's device address (do it before any
 * stream capture). Calls that overlap on the GPU (two streams at once) share the array and race.
 * cfg: the configuration the state belongs to (physical constants). in: device pointers.
 * dev_out5: device double[5] receiving kinetic_ion, kinetic_electron, field_E, field_B, pair
 * (J per metre of y). Work is queued on stream; the call does not synchronise. Refuses (PIC_EINVAL)
 * particle counts above 2^31 - 1, grids outside 3 <= nx, 4 <= nz < 32768, missing pointers and
 * a pot_mode outside 0..2 (2 without 0 < morse_a < 1000). */
PIC_API int pic_energy_noalloc(const pic_config* cfg, const pic_state_view* in, double* dev_out5, void* stream);

/* ---- checkpoint / resume ------------------------------------------------------------------
 * A checkpoint is a caller-owned buffer of pic_checkpoint_size bytes, in device memory (256-byte
 * aligned) or host memory (on_host != 0; pinned memory makes the copies faster), holding the
 * particles, tile offsets, fields, node density, current, the injected-energy sum and the step
 * counter of a context. Restoring it into the same context, or into a new context made from the
 * same configuration (another process, after writing the host buffer to disk), resumes bit for
 * bit: same grids, same particle set (a cell sort after the restore may order the particles of
 * one cell differently). A device save is asynchronous on the context's stream; a host save and
 * every restore synchronise. pic_checkpoint_restore returns PIC_EINVAL for a buffer that holds no
 * checkpoint of this layout. */
PIC_API int pic_checkpoint_size(pic_ctx* ctx, size_t* bytes);
PIC_API int pic_checkpoint_save(pic_ctx* ctx, void* buf, int32_t on_host);
PIC_API int pic_checkpoint_restore(pic_ctx* ctx, const void* buf, int32_t on_host);

/* ---- differentiable cycle (2D, sort_every = 0, pot_mode 0) ----------------------------------
 * Gradients of L = sum_nodes w(node) n(node)/n0 (pair-species density at the final state)
 *                 + kin * (total kinetic energy of all species, J per metre of y)
 * with respect to the pair-potential parameters D (J) and r0 (m) and, in PIC_MODE_FULL, the laser
 * peak intensity I0 (W/m^2), by hand-written FP64 adjoint kernels of the step. In
 * PIC_MODE_TRANSPORT the step is node density -> Eqs. (1)-(3) force -> kick -> move; in
 * PIC_MODE_FULL it is the whole cycle: density, pair force, staggered E/B gather, Boris push,
 * move, walls, charge-conserving current, Yee update with Mur walls and the antenna (E0 =
 * sqrt(2 I0 / (eps0 c)) scales the source). The fixed-point deposition and current are
 * differentiated as the continuous linear shape. The paper has no adjoint; the method, the
 * parameters and the stage are the paper's.
 *
 * Adjoint buffers (device, caller-owned). Per-particle adjoints and the particles' scatter onto
 * the nodes are FP32 (the precision of the push), field adjoints and parameter derivatives FP64:
 *   lam_pos[s]: float, 2 n_s, (x, z) adjoints per particle of species s (per cell), in the
 *               context's particle order;
 *   lam_u[s]:   float, 3 n_s;
 *   lam_nodes:  float, (nz+1) nx scratch;
 *   lam_F:      double, 9 (nz+1) nx: adjoints of Ex Ey Ez Bx By Bz and three scratch grids (FULL only);
 *   lam_j:      float, 3 (nz+1) nx scratch (FULL only);
 *   grads:      double, 3, accumulated by pic_adjoint_step: dL/dD (1/J), dL/dr0 (1/m), dL/dI0 (m^2/W).
 * Unused pointers (second species, FULL-only buffers in transport mode) may be NULL.
 *
 * pic_node_functional: *host_out = sum_nodes w n/n0 at the current state (w: device double
 *   (nz+1)*nx, e.g. a crater-depth weighting).
 * pic_adjoint_seed: at the final state, set the adjoints of the loss (momenta: kin w m c^2 u/gamma,
 *   positions: the gradient of the density functional, fields: 0); *host_dLdr0 receives the r0
 *   derivative of the density unit in the functional (add it to grads[1]).
 * pic_adjoint_step: with the context at the state of step t (restore it from a checkpoint), map the
 *   adjoints of step t+1 to step t in place and add this step's parameter derivatives to grads.
 * Both return PIC_ESTATE outside 2D, sort_every = 0 and pot_mode 0. */
typedef struct {
    float* lam_pos[2];
    float* lam_u[2];
    float* lam_nodes;
    double* lam_F;
    float* lam_j;
    double* grads;
} pic_adjoint_buffers;

PIC_API int pic_node_functional(pic_ctx* ctx, const double* dev_weights, double* host_out);
PIC_API int pic_adjoint_seed(pic_ctx* ctx, double kin, const double* dev_weights, const pic_adjoint_buffers* bufs,
                             double* host_dLdr0);
PIC_API int pic_adjoint_step(pic_ctx* ctx, const pic_adjoint_buffers* bufs);

/* Static text for a return code. */
PIC_API const char* pic_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
