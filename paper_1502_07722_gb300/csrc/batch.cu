// Batched intensity sweep: several independent slabs (uneven sizes, particle counts and laser
// intensities) advanced together. Each slab is an ordinary context (pic_init on a slice of the
// batch workspace); a step of the whole batch is
//   k_prepare_batch      clear the currents, start the next node density from the current one
//   k_particles_batch    one persistent launch over the tiles of every slab
//   field kernels        one launch each for all slabs (blockIdx.z = slab), antenna on the device
// and is recorded once as a CUDA graph per parity of the double-buffered node density, then
// replayed. The per-slab arguments live in device memory (copied into a constant-memory table in
// front of the particle kernel), so a cell sort (host-driven, every
// sort_every steps) only refreshes them; the graphs stay valid.
#include <cstring>
#include <new>
#include <vector>

#include "pic_internal.cuh"

namespace gbpic {
void sort_species_impl(Ctx& c, int s, cudaStream_t st, int from_b, int64_t* launches);
int max_batch_slabs();

constexpr int kMaxSlabs = 48;    // the constant-memory argument table of the batched particle kernel
static_assert(kMaxSlabs <= kMaxFieldSlabs, "every slab's field arguments fit the batched field kernels' parameters");

__global__ void k_prepare_batch(const StepArgs* __restrict__ args)
{
    const StepArgs& a = args[blockIdx.y];
    const size_t nn = (size_t)(a.nz + 1) * a.nx;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nn; j += (size_t)gridDim.x * blockDim.x) {
        a.J[0][j] = 0;
        a.J[1][j] = 0;
        a.J[2][j] = 0;
        a.rho_next[j] = a.rho_cur[j];
    }
}

}  // namespace gbpic

using namespace gbpic;

struct pic_batch {
    int n;
    pic_ctx* slab[kMaxSlabs];
    cudaStream_t st;
    int full, pot, maxW, max_nx, max_nz, total_tiles, nsm, sort_every, steps_since_sort;
    size_t max_nn;
    int64_t step;
    StepArgs* args_dev;          // [2][n]: parity 0 (density in buffer 0) and parity 1
    FieldBatch fields;           // every slab's field arguments (host copy, passed by value)
    AntennaParams* ap_dev;       // [n]
    long long* step_dev;         // [n]
    float* ant_dev;              // [n][2]
    int* tile_base_dev;          // [n + 1]
    cudaGraphExec_t graph[2];
    int captured;
    int timing;
    cudaEvent_t ev[6];
    double ms[3];
    int64_t nlaunch[4];
    int sticky;
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t batch_tail_bytes(int n)
{
    return a256(sizeof(StepArgs) * 2 * n) + a256(sizeof(AntennaParams) * n) + a256(8 * (size_t)n) +
           a256(8 * (size_t)n) + a256(4 * ((size_t)n + 1));
}

int upload_args(pic_batch* b)
{
    std::vector<StepArgs> h(2 * b->n);
    for (int s = 0; s < b->n; s++) {
        Ctx& c = b->slab[s]->c;
        const int cur = c.cur;
        for (int p = 0; p < 2; p++) {
            c.cur = p;
            h[p * b->n + s] = make_step_args(c);
        }
        c.cur = cur;
    }
    if (cudaMemcpyAsync(b->args_dev, h.data(), sizeof(StepArgs) * h.size(), cudaMemcpyHostToDevice, b->st) !=
        cudaSuccess)
        return PIC_ECUDA;
    return cudaStreamSynchronize(b->st) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

void enqueue_step(pic_batch* b, int parity)
{
    const StepArgs* args = b->args_dev + parity * b->n;
    dim3 pg((unsigned)((b->max_nn + 1023) / 1024 > 4096 ? 4096 : (b->max_nn + 1023) / 1024), b->n);
    k_prepare_batch<<<pg, 256, 0, b->st>>>(args);
    if (b->timing) cudaEventRecord(b->ev[0], b->st);
    launch_particle_step_batch(args, b->tile_base_dev, b->n, b->total_tiles, b->full, b->pot, b->maxW, b->nsm, b->st);
    if (b->timing) cudaEventRecord(b->ev[1], b->st);
    if (b->full)
        launch_fields_batch(b->fields, b->ap_dev, b->step_dev, b->ant_dev, b->st);
    if (b->timing) cudaEventRecord(b->ev[2], b->st);
}

int capture(pic_batch* b)
{
    for (int p = 0; p < 2; p++) {
        cudaGraph_t g;
        if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PIC_ECUDA;
        enqueue_step(b, p);
        if (cudaStreamEndCapture(b->st, &g) != cudaSuccess) return PIC_ECUDA;
        const cudaError_t e = cudaGraphInstantiate(&b->graph[p], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return PIC_ECUDA;
    }
    b->captured = 1;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_workspace_size(const pic_config* cfgs, int32_t n, size_t* bytes)
{
    if (!cfgs || !bytes || n < 1 || n > kMaxSlabs) return PIC_EINVAL;
    size_t t = 0;
    for (int s = 0; s < n; s++) {
        if (cfgs[s].mode != cfgs[0].mode || (cfgs[s].dims != 0 && cfgs[s].dims != 2)) return PIC_EINVAL;
        if (cfgs[s].pot_mode != cfgs[0].pot_mode || cfgs[s].lattice != cfgs[0].lattice)
            return PIC_EINVAL;   // one kernel instance
        size_t b = 0;
        const int r = pic_workspace_size(&cfgs[s], &b);
        if (r) return r;
        t += a256(b);
    }
    *bytes = t + batch_tail_bytes(n);
    return PIC_OK;
}

int pic_batch_init(const pic_config* cfgs, int32_t n, void* workspace, size_t bytes, void* stream, pic_batch** out)
{
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    size_t need = 0;
    int r = pic_batch_workspace_size(cfgs, n, &need);
    if (r) return r;
    if (!workspace || ((uintptr_t)workspace & 255) || !stream) return PIC_EINVAL;
    if (bytes < need) return PIC_ENOMEM;
    pic_batch* b = new (std::nothrow) pic_batch();
    if (!b) return PIC_ENOMEM;
    b->n = n;
    b->st = (cudaStream_t)stream;
    char* p = (char*)workspace;
    std::vector<int> tile_base(n + 1, 0);
    for (int s = 0; s < n; s++) {
        size_t sb = 0;
        pic_workspace_size(&cfgs[s], &sb);
        r = pic_init(&cfgs[s], p, sb, stream, &b->slab[s]);
        if (r) {
            for (int q = 0; q < s; q++) pic_free(b->slab[q]);
            delete b;
            return r;
        }
        b->slab[s]->c.in_batch = 1;
        p += a256(sb);
        const Ctx& c = b->slab[s]->c;
        tile_base[s + 1] = tile_base[s] + c.ntiles;
        b->maxW = c.W > b->maxW ? c.W : b->maxW;
        b->max_nx = c.nx > b->max_nx ? c.nx : b->max_nx;
        b->max_nz = c.nz > b->max_nz ? c.nz : b->max_nz;
        b->max_nn = c.nn > b->max_nn ? c.nn : b->max_nn;
        b->nsm = c.nsm;
    }
    b->total_tiles = tile_base[n];
    b->full = cfgs[0].mode == PIC_MODE_FULL;
    b->pot = pot_code(cfgs[0]);   // kernel instance
    b->sort_every = cfgs[0].sort_every;
    b->args_dev = reinterpret_cast<StepArgs*>(p);
    p += a256(sizeof(StepArgs) * 2 * n);
    b->ap_dev = reinterpret_cast<AntennaParams*>(p);
    p += a256(sizeof(AntennaParams) * n);
    b->step_dev = reinterpret_cast<long long*>(p);
    p += a256(8 * (size_t)n);
    b->ant_dev = reinterpret_cast<float*>(p);
    p += a256(8 * (size_t)n);
    b->tile_base_dev = reinterpret_cast<int*>(p);
    std::vector<AntennaParams> ap(n);
    b->fields.n = n;
    for (int s = 0; s < n; s++) {
        b->fields.f[s] = make_field_args(b->slab[s]->c);
        b->fields.f[s].ant = b->ant_dev + 2 * s;     // the batch's per-slab antenna scalars
        ap[s] = make_antenna_params(b->slab[s]->c);
    }
    field_row_blocks(b->fields);
    bool ok = cudaMemcpyAsync(b->ap_dev, ap.data(), sizeof(AntennaParams) * n, cudaMemcpyHostToDevice, b->st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->tile_base_dev, tile_base.data(), 4 * (size_t)(n + 1), cudaMemcpyHostToDevice,
                              b->st) == cudaSuccess &&
              cudaMemsetAsync(b->step_dev, 0, 8 * (size_t)n, b->st) == cudaSuccess;
    r = ok ? upload_args(b) : PIC_ECUDA;
    for (int q = 0; q < 6 && r == PIC_OK; q++)
        if (cudaEventCreate(&b->ev[q]) != cudaSuccess) r = PIC_ECUDA;
    if (r) {
        for (int q = 0; q < n; q++) pic_free(b->slab[q]);
        delete b;
        return r;
    }
    *out = b;
    return PIC_OK;
}

void pic_batch_free(pic_batch* b)
{
    if (!b) return;
    for (int p = 0; p < 2; p++)
        if (b->captured) cudaGraphExecDestroy(b->graph[p]);
    for (int q = 0; q < 6; q++)
        if (b->ev[q]) cudaEventDestroy(b->ev[q]);
    for (int s = 0; s < b->n; s++) pic_free(b->slab[s]);
    delete b;
}

int pic_batch_slab(pic_batch* b, int32_t i, pic_ctx** out)
{
    if (!b || !out || i < 0 || i >= b->n) return PIC_EINVAL;
    *out = b->slab[i];
    return PIC_OK;
}

int pic_batch_step(pic_batch* b, int32_t nsteps)
{
    if (!b || nsteps < 0) return PIC_EINVAL;
    if (b->sticky) return b->sticky;
    for (int it = 0; it < nsteps; it++) {
        if (b->sort_every > 0 && b->steps_since_sort >= b->sort_every) {
            if (b->timing) cudaEventRecord(b->ev[3], b->st);
            for (int s = 0; s < b->n; s++) {
                Ctx& c = b->slab[s]->c;
                for (int sp = 0; sp < c.nsp; sp++) sort_species_impl(c, sp, b->st, 0, &b->nlaunch[2]);
            }
            if (b->timing) {
                cudaEventRecord(b->ev[4], b->st);
                cudaEventSynchronize(b->ev[4]);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, b->ev[3], b->ev[4]);
                b->ms[2] += ms;
            }
            const int r = upload_args(b);      // the sort swapped the particle buffers
            if (r) return r;
            b->steps_since_sort = 0;
        }
        const int parity = b->slab[0]->c.cur;
        if (b->timing) {
            // direct launches with events around the particle kernel and the field kernels
            enqueue_step(b, parity);
            if (cudaEventSynchronize(b->ev[2]) != cudaSuccess) return PIC_ECUDA;
            float m0 = 0.f, m1 = 0.f;
            cudaEventElapsedTime(&m0, b->ev[0], b->ev[1]);
            cudaEventElapsedTime(&m1, b->ev[1], b->ev[2]);
            b->ms[0] += m0;
            b->ms[1] += m1;
            b->nlaunch[0] += 1;
            b->nlaunch[1] += b->full ? 6 : 0;
            b->nlaunch[3] += 2 + (b->full ? 6 : 0);
        } else {
            if (!b->captured) {
                const int r = capture(b);
                if (r) return r;
            }
            if (cudaGraphLaunch(b->graph[parity], b->st) != cudaSuccess) return PIC_ECUDA;
            b->nlaunch[3] += 2 + (b->full ? 6 : 0);
        }
        for (int s = 0; s < b->n; s++) {
            Ctx& c = b->slab[s]->c;
            c.cur = 1 - c.cur;
            c.step++;
        }
        b->step++;
        b->steps_since_sort++;
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(b->st) != cudaSuccess) return PIC_ECUDA;
    for (int s = 0; s < b->n; s++) {
        Ctx& c = b->slab[s]->c;
        unsigned stw = 0;
        if (cudaMemcpy(&stw, c.status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
        if (stw & kErrNan) c.sticky = PIC_ENAN;
        else if (stw & kErrMove) c.sticky = PIC_EMOVE;
        else if (stw & kErrOverflow) c.sticky = PIC_EOVERFLOW;
        if (c.sticky && !b->sticky) b->sticky = c.sticky;
    }
    return b->sticky;
}

int pic_batch_set_timing(pic_batch* b, int32_t enable)
{
    if (!b) return PIC_EINVAL;
    b->timing = enable != 0;
    for (int q = 0; q < 3; q++) b->ms[q] = 0.0;
    for (int q = 0; q < 4; q++) b->nlaunch[q] = 0;
    return PIC_OK;
}

int pic_batch_get_timing(pic_batch* b, double ms[3], int64_t n[4])
{
    if (!b || !ms || !n) return PIC_EINVAL;
    for (int q = 0; q < 3; q++) ms[q] = b->ms[q];
    for (int q = 0; q < 4; q++) n[q] = b->nlaunch[q];
    return PIC_OK;
}

}  // extern "C"
