// Cell sort of one species into tiles (counting sort by a tile-major cell key):
// count per key -> exclusive scan -> scatter into the second buffer -> swap.
// The key of cell (i, k) is tile * T^2 + (k mod T) * T + (i mod T), tile = (k / T) * ntx + i / T
// (in 3D likewise with T^3 cells per tile), so the particles of a tile are contiguous.
// Inside a tile the cell-ordered list is cut into blocks of kLayoutBlock particles (1024 in 2D,
// 256 in 3D: 32 x the particles per cell of a typical slab) and each block is stored column by
// column as a 32-row matrix whose rows are consecutive runs of the cell order. The particle
// kernels read their records in memory order, coalesced, and the 32 lanes of a warp then hold
// particles one run apart: neighbouring cells, so a warp's deposits go to distinct nodes that
// share cache sectors, without a transposing copy through shared memory.
// The order of particles inside one cell is not fixed (atomic cursors); nothing downstream
// depends on it because every deposit is an exact integer sum.
#include <cmath>

#include "pic_internal.cuh"

namespace gbpic {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 2 * kScanBlock;

// Division by a run-time divisor d >= 1 for 0 <= x < 2^31: q = umulhi(x, m) with m = floor((2^32 - 1) / d)
// is at most one short of x / d (x m / 2^32 > x / d - x (1 + 1/d) / 2^32 > x / d - 1), so one
// correction makes it exact.
struct Div {
    int d;
    unsigned m;
};
inline Div make_div(int d) { return Div{d, (unsigned)(4294967295ULL / (unsigned long long)d)}; }
__device__ __forceinline__ int divq(int x, Div D, int& r)
{
    unsigned q = __umulhi((unsigned)x, D.m);
    int rr = x - (int)q * D.d;
    if (rr >= D.d) {
        q++;
        rr -= D.d;
    }
    r = rr;
    return (int)q;
}

struct KeyGeo {
    int nx, ny, T, ntx, nty, dims;
    int TT;     // cells per tile
    Div dnx, dny, dT, dTT;
};

constexpr int kLayoutBlock2 = 1024, kLayoutBlock3 = 256;

// Storage slot, relative to its tile, of the particle at place ci of the tile's cell order (nt
// particles in the tile): block ci / B, and inside a block of nb particles the element (row
// j / C, column j mod C) of a row-major matrix with C = ceil(nb / 32) columns, stored column-major
// (the last row may be short, so column c holds R + (c < rem) elements). A bijection of 0..nt-1.
template <int B>
__device__ __forceinline__ int layout_slot(int ci, int nt)
{
    const int blk = ci / B, j = ci - blk * B, nb = min(B, nt - blk * B);
    if (nb == B) {
        // a full block: B / 32 columns of 32 (shifts)
        constexpr int C = B / 32;
        return blk * B + (j % C) * 32 + j / C;
    }
    const int C = (nb + 31) >> 5, R = nb / C, rem = nb - R * C;
    const int r = j / C, c = j - r * C;
    return blk * B + c * R + min(c, rem) + r;
}

// 2D: cell = k*nx + i; 3D: cell = (k*ny + j)*nx + i. Tiles of T^dims cells, tile-major.
__device__ __forceinline__ int cell_key(int cell, const KeyGeo& g)
{
    int i, j = 0, li, lj, lk;
    const int q = divq(cell, g.dnx, i);
    int k = q;
    if (g.dims == 3) k = divq(q, g.dny, j);
    const int tx = divq(i, g.dT, li), tz = divq(k, g.dT, lk);
    if (g.dims == 2) return (tz * g.ntx + tx) * g.TT + lk * g.T + li;
    const int ty = divq(j, g.dT, lj);
    const int tile = (tz * g.nty + ty) * g.ntx + tx;
    return ((tile * g.T + lk) * g.T + lj) * g.T + li;
}

// Count the particles of every key. The sort's block layout stores B cell-ordered particles as a
// 32-row matrix column by column, so storage slot c * 32 + r holds cell-order place r * (B / 32) + c:
// a lane that walks its warp's chunk of B slots with stride 32 meets consecutive particles of the
// cell order (between sorts they have barely moved) and issues one atomic per run of equal keys
// instead of one per particle (any order stays correct; only the runs get shorter).
__global__ void k_count(const int32_t* __restrict__ cell, int64_t n, KeyGeo kg, int32_t* count, int cols)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5, chunk = 32 * (int64_t)cols;
    for (int64_t base = warp * chunk; base < n; base += nwarp * chunk) {
        int key = -1, run = 0;
        for (int c = 0; c < cols; c++) {
            const int64_t p = base + 32 * (int64_t)c + lane;
            if (p >= n) break;
            const int k = cell_key(cell[p], kg);
            if (k != key) {
                if (run) atomicAdd(count + key, run);
                key = k;
                run = 0;
            }
            run++;
        }
        if (run) atomicAdd(count + key, run);
    }
}

// exclusive scan of kScanItems elements per block; block totals to bsum
__global__ void k_scan_block(const int32_t* __restrict__ in, int32_t* out, int32_t* bsum, int n)
{
    __shared__ int32_t s[kScanItems];
    const int base = blockIdx.x * kScanItems;
    for (int j = threadIdx.x; j < kScanItems; j += blockDim.x) s[j] = base + j < n ? in[base + j] : 0;
    __syncthreads();
    // Blelloch up-sweep / down-sweep
    int off = 1;
    for (int d = kScanItems >> 1; d > 0; d >>= 1) {
        __syncthreads();
        if ((int)threadIdx.x < d) {
            const int ai = off * (2 * threadIdx.x + 1) - 1, bi = off * (2 * threadIdx.x + 2) - 1;
            s[bi] += s[ai];
        }
        off <<= 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = s[kScanItems - 1];
        s[kScanItems - 1] = 0;
    }
    for (int d = 1; d < kScanItems; d <<= 1) {
        off >>= 1;
        __syncthreads();
        if ((int)threadIdx.x < d) {
            const int ai = off * (2 * threadIdx.x + 1) - 1, bi = off * (2 * threadIdx.x + 2) - 1;
            const int32_t t = s[ai];
            s[ai] = s[bi];
            s[bi] += t;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kScanItems; j += blockDim.x)
        if (base + j < n) out[base + j] = s[j];
}

// exclusive scan of the block totals in place (one block, sequential over chunks)
__global__ void k_scan_sums(int32_t* bsum, int nb)
{
    __shared__ int32_t s[kScanBlock];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanBlock) {
        const int j = base + threadIdx.x;
        const int32_t v = j < nb ? bsum[j] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < kScanBlock; d <<= 1) {     // Hillis-Steele inclusive
            const int32_t t = (int)threadIdx.x >= d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (j < nb) bsum[j] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += s[kScanBlock - 1];
        __syncthreads();
    }
}

__global__ void k_scan_add(int32_t* out, const int32_t* __restrict__ bsum, int n, int32_t* cursor, int32_t total)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        const int32_t v = out[j] + bsum[j / kScanItems];
        out[j] = v;
        cursor[j] = v;
    }
    if (j == 0) out[n] = total;
}

// Key of cell (i, j, k) (j = 0 in 2D), as cell_key computes it from the cell index.
__device__ __forceinline__ int key_of(int i, int j, int k, const KeyGeo& g)
{
    int li, lj, lk;
    const int tx = divq(i, g.dT, li), tz = divq(k, g.dT, lk);
    if (g.dims == 2) return (tz * g.ntx + tx) * g.TT + lk * g.T + li;
    const int ty = divq(j, g.dT, lj);
    const int tile = (tz * g.nty + ty) * g.ntx + tx;
    return ((tile * g.T + lk) * g.T + lj) * g.T + li;
}

// The largest particle count (of one species) over the blocks of 4 cells per axis (x, y periodic;
// blocks reaching past the last row of cells are cut there): the particles that can reach one
// node in a step sit in such a block. Two passes: the counts copied from key order into cell order,
// then a separable sum: a CTA owns a TX x TY patch of columns (i, j) and a segment of KZ rows; it
// walks the rows (plus the three above the segment), forms each row's 4 x KY sums from a
// shared-memory copy of the patch with its halo, keeps the last three rows' sums in registers and
// closes the block of base row k - 3 at row k. One atomicMax per warp into *out. (The direct
// form, 4^dims key lookups per cell, took 1.9 ms per species on the 384^2 x 256 slab.)
__global__ void k_counts_to_cells(const int32_t* __restrict__ count, KeyGeo kg, int nz, int32_t* out)
{
    const int64_t ncell = (int64_t)kg.nx * kg.ny * nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += stride) {
        int i, j;
        const int q = divq((int)c, kg.dnx, i);
        const int k = divq(q, kg.dny, j);
        out[c] = count[key_of(i, j, k, kg)];
    }
}

constexpr int kMaxRows = 64;      // rows of cells per CTA of k_block_max

template <int TX, int TY, int KY>
__global__ void __launch_bounds__(TX * TY) k_block_max(const int32_t* __restrict__ cc, int nx, int ny, int nz,
                                                        unsigned* out)
{
    __shared__ int32_t s[TY + KY - 1][TX + 3];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * kMaxRows;
    const bool own = i0 + tx < nx && j0 + ty < ny;
    const int kend = min(k0 + kMaxRows + 3, nz);
    unsigned r0 = 0, r1 = 0, r2 = 0, m = 0;      // sums of rows k - 3, k - 2, k - 1
    for (int k = k0; k < kend; k++) {
        __syncthreads();
        for (int q = threadIdx.x; q < (TY + KY - 1) * (TX + 3); q += TX * TY) {
            const int b = q / (TX + 3), a = q - b * (TX + 3);
            s[b][a] = cc[((size_t)k * ny + (j0 + b) % ny) * nx + (i0 + a) % nx];
        }
        __syncthreads();
        unsigned p = 0;
#pragma unroll
        for (int dj = 0; dj < KY; dj++)
#pragma unroll
            for (int di = 0; di < 4; di++) p += (unsigned)s[ty + dj][tx + di];
        if (k - 3 >= k0) m = max(m, r0 + r1 + r2 + p);
        r0 = r1;
        r1 = r2;
        r2 = p;
    }
    if (kend == nz) {
        // the blocks cut at the last row, base rows nz - 3 .. nz - 1 of this segment
        if (nz - 3 >= k0 && nz - 3 < k0 + kMaxRows) m = max(m, r0 + r1 + r2);
        if (nz - 2 >= k0 && nz - 2 < k0 + kMaxRows) m = max(m, r1 + r2);
        if (nz - 1 >= k0 && nz - 1 < k0 + kMaxRows) m = max(m, r2);
    }
    if (!own) m = 0;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

static int64_t ncell_blocks(const Ctx& c)
{
    const int64_t ncell = (int64_t)c.nx * c.ny * c.nz;
    return (ncell + 255) / 256 > 0 ? (ncell + 255) / 256 : 1;
}

// Fixed-point range: every int64 node sum is exact while the particles that can reach one node
// (both species: bounded by the sum of the two species' largest block counts from their last
// sorts) stay within the limit the context was set up for; beyond it the sticky overflow bit is
// raised.
__global__ void k_count_check(unsigned* status, long long limit)
{
    if (threadIdx.x == 0 && (long long)status[4] + (long long)status[5] > limit) atomicOr(status, kErrOverflow);
}

__global__ void k_tile_starts(const int32_t* __restrict__ off, int ntiles, int TT, int32_t* tile_start)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= ntiles) tile_start[t] = off[(size_t)t * TT];
}

__global__ void k_scatter(SpeciesBuf src, SpeciesBuf dst, int64_t n, KeyGeo kg, int32_t* cursor,
                          const int32_t* __restrict__ tile_start)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (n + 31) & ~(int64_t)31;
    const unsigned lane = threadIdx.x & 31;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nround; p += stride) {
        const bool valid = p < n;
        const int c = valid ? src.cell[p] : 0;
        const int key = valid ? cell_key(c, kg) : -1;
        // one cursor atomic per distinct key in the warp; lanes take consecutive slots
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (valid && (int)lane == leader) base = atomicAdd(cursor + key, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (!valid) continue;
        // place in the cell order -> storage slot of the tile's block layout
        int kt;
        const int t = divq(key, kg.dTT, kt), ts = tile_start[t];
        const int ci = base + __popc(peers & ((1u << lane) - 1u)) - ts, nt = tile_start[t + 1] - ts;
        const int q = ts + (kg.dims == 3 ? layout_slot<kLayoutBlock3>(ci, nt) : layout_slot<kLayoutBlock2>(ci, nt));
        dst.cell[q] = c;
        dst.fx[q] = src.fx[p];
        if (kg.dims == 3) dst.fy[q] = src.fy[p];
        dst.fz[q] = src.fz[p];
        dst.ux[q] = src.ux[p];
        dst.uy[q] = src.uy[p];
        dst.uz[q] = src.uz[p];
    }
}

// Sort species s: its particles are read from `b` when from_b != 0 (fresh data), else from `a`;
// the sorted result always ends in `a`.
void sort_species_impl(Ctx& c, int s, cudaStream_t st, int from_b, int64_t* launches)
{
    Species& S = c.sp[s];
    const int TT = c.dims == 3 ? c.T * c.T * c.T : c.T * c.T;
    const KeyGeo kg = {c.nx, c.ny, c.T, c.ntx, c.nty, c.dims, TT, make_div(c.nx), make_div(c.ny), make_div(c.T),
                       make_div(TT)};
    int64_t g = (S.n + 255) / 256;
    if (g > (int64_t)c.nsm * 16) g = (int64_t)c.nsm * 16;
    if (g < 1) g = 1;
    cudaMemsetAsync(c.keys_count, 0, sizeof(int32_t) * (size_t)(c.nkeys + 1), st);
    cudaMemsetAsync(c.status + 4 + s, 0, sizeof(unsigned), st);
    SpeciesBuf src = from_b ? S.b : S.a;
    SpeciesBuf dst = from_b ? S.a : S.b;
    if (S.n > 0)
        k_count<<<(int)g, 256, 0, st>>>(src.cell, S.n, kg, c.keys_count,
                                        (c.dims == 3 ? kLayoutBlock3 : kLayoutBlock2) / 32);
    const int nb = (c.nkeys + kScanItems - 1) / kScanItems;
    // the most particles of this species in one block of 4 cells per axis (counts are consumed
    // below; the key offsets, written by the scan after it, hold the counts in cell order meanwhile)
    k_counts_to_cells<<<(int)(ncell_blocks(c) < (int64_t)c.nsm * 16 ? ncell_blocks(c) : (int64_t)c.nsm * 16), 256, 0,
                        st>>>(c.keys_count, kg, c.nz, c.keys_off);
    const unsigned zs = (unsigned)((c.nz + kMaxRows - 1) / kMaxRows);
    if (c.dims == 3)
        k_block_max<32, 8, 4><<<dim3((unsigned)((c.nx + 31) / 32), (unsigned)((c.ny + 7) / 8), zs), 256, 0, st>>>(
            c.keys_off, c.nx, c.ny, c.nz, c.status + 4 + s);
    else
        k_block_max<256, 1, 1><<<dim3((unsigned)((c.nx + 255) / 256), 1u, zs), 256, 0, st>>>(c.keys_off, c.nx, 1, c.nz,
                                                                                           c.status + 4 + s);
    k_scan_block<<<nb, kScanBlock, 0, st>>>(c.keys_count, c.keys_off, c.scan_tmp, c.nkeys);
    k_scan_sums<<<1, kScanBlock, 0, st>>>(c.scan_tmp, nb);
    // the cursor reuses the count array (counts are consumed by the scan)
    k_scan_add<<<(c.nkeys + 255) / 256, 256, 0, st>>>(c.keys_off, c.scan_tmp, c.nkeys, c.keys_count, (int32_t)S.n);
    k_tile_starts<<<(c.ntiles + 1 + 255) / 256, 256, 0, st>>>(c.keys_off, c.ntiles, TT, S.tile_start);
    if (S.n > 0) k_scatter<<<(int)g, 256, 0, st>>>(src, dst, S.n, kg, c.keys_count, S.tile_start);
    k_count_check<<<1, 32, 0, st>>>(c.status, c.count_limit);
    if (!from_b) {
        SpeciesBuf t = S.a;
        S.a = S.b;
        S.b = t;
    }
    if (launches) *launches += 7 + (S.n > 0 ? 2 : 0);
}

void launch_sort_species(Ctx& c, int s, cudaStream_t st, int64_t* launches)
{
    sort_species_impl(c, s, st, 0, launches);
}

// Largest contribution of one particle to one node sum (a particle's stencil starts at the lower of
// its old and new cells and spans 3 nodes per axis, so a node collects from a block of 4 cells per
// axis):
//   2D J6y: |V| W6 <= 2^b * 6 * 2^32 (|beta_y| < 1; W6 = 2 S0xS0z + S1xS0z + S0xS1z + 2 S1xS1z);
//   2D J2x, J2z: <= 2 * 2^16 * 2^17 = 2^34 (prefix sums of dS * (S0 + S1));
//   2D density: weight products <= 2^32, old and new positions both counted while the kernel updates
//   the sum incrementally: 2^33;
//   3D currents: <= 2 * 2^14 * 6 * 2^28 = 3 * 2^44; 3D density 2 * 2^42.
// A node sum stays below 2^63 while the particles of one block (both species) number fewer than
// 2^63 / (largest contribution): the limit returned (particles per block of 4^dims cells).
int64_t count_limit(int dims, int full, int jy_bits)
{
    const double two63 = 9223372036854775808.0;
    double lim;
    if (dims == 3) {
        lim = two63 / (2.0 * 4398046511104.0);                                     // density
        if (full) lim = fmin(lim, two63 / (3.0 * 17592186044416.0));              // currents
    } else {
        lim = two63 / (2.0 * 4294967296.0);                                        // density
        if (full) {
            lim = fmin(lim, two63 / 17179869184.0);                                // J2x, J2z
            lim = fmin(lim, two63 / (6.0 * 4294967296.0 * ldexp(1.0, jy_bits)));  // J6y
        }
    }
    return (int64_t)floor(lim - 1e-9);
}

// The J_y code resolution: 2^18 unless a uniform slab of n particles per cell (16 n per block, with
// a quarter headroom for compression) could overflow J6y at that resolution; then the largest b
// whose limit holds them.
int choose_jy_bits(int64_t n_per_cell)
{
    for (int b = 18; b >= 1; b--)
        if ((double)count_limit(2, 1, b) >= 1.25 * 16.0 * (double)n_per_cell) return b;
    return 0;
}

}  // namespace gbpic
