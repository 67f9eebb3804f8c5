// api.cu -- context and workspace, status strings, device scan and stable
// radix sort utilities, the target normal map and the Eq. (1) warp.
#include <stdlib.h>
#include <string.h>

#include "ed_internal.cuh"

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------

namespace {

struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

void normalise_limits(ed_limits &L)
{
    if (L.max_pairs_per_node <= 0) L.max_pairs_per_node = 48;
    if (L.max_cells <= 0) L.max_cells = 1 << 22;
}

size_t carve(ed_context *c, char *base)
{
    const ed_limits &L = c->lim;
    const size_t N = (size_t)L.max_points, M = (size_t)L.max_nodes;
    const size_t WH = (size_t)L.max_width * L.max_height;
    const size_t cells = (size_t)L.max_cells;
    const size_t nnzb = M * (size_t)L.max_pairs_per_node;
    const size_t nent = 10 * N;
    const size_t tiles = (nent + 1023) / 1024 + 1;
    const size_t P = 12 * M + 6;
    const size_t big = (N > WH ? N : WH);
    size_t scan_len = big > 256 * tiles ? big : 256 * tiles;
    if (nnzb > scan_len) scan_len = nnzb;
    if (cells + 1 > scan_len) scan_len = cells + 1;   // node flags over the sampling grid
    Carver k{base};
    c->misc = k.take<int>(MI_COUNT);
    c->fmisc = k.take<float>(MF_COUNT);
    c->dmisc = k.take<double>(64);
    c->cell_of = k.take<int>(N);
    c->cell_pick = k.take<int>(cells);
    c->cell_node = k.take<int>(cells);
    c->kcell_start = k.take<int>(cells + 1);
    c->kcell_cnt = k.take<int>(cells + 1);
    c->kcell_pos = k.take<float4>(M);
    c->bm_words = (int)((M + 31) / 32);
    c->bitmap = k.take<uint32_t>(M * (size_t)c->bm_words);
    c->row_ptr = k.take<int>(M + 1);
    c->row_cnt = k.take<int>(M + 1);
    c->col = k.take<int>(nnzb);
    c->brow = k.take<int>(nnzb);
    c->tpos = k.take<int>(nnzb);
    c->diag_pos = k.take<int>(M);
    c->up_list = k.take<int>(nnzb);
    c->fin_info = k.take<int4>(2 * ((nnzb + M) / 2 + 1));
    c->max_nnzb = (int)nnzb;
    c->ent_key = k.take<uint32_t>(nent);
    c->ent_val = k.take<uint32_t>(nent);
    c->ent_key2 = k.take<uint32_t>(nent);
    c->ent_val2 = k.take<uint32_t>(nent);
    c->radix_cnt = k.take<int>(256 * tiles + 1);
    c->inc = k.take<uint32_t>(nent);
    c->ent_start = k.take<int>(nnzb + 1);
    c->perm = k.take<int>(N);
    c->spos = k.take<float4>(N);
    c->snrm = k.take<float4>(N);
    c->sidx = k.take<ushort4>(N);
    c->sw = k.take<float4>(N);
    c->sidx_d = k.take<ushort4>(N);
    c->sw_d = k.take<float4>(N);
    c->run_start = k.take<int>(N + 1);
    c->run_of_start = k.take<int>(N);
    c->bcnt = k.take<int>(2 * (M + 1));
    c->bstart = k.take<int>(M + 1);
    c->icnt = k.take<int>(2 * (nnzb + 1) + 2 * ED_ASM_BINS);
    c->asm_bins = c->icnt + 2 * (nnzb + 1);
    c->crec0 = k.take<float4>(N);
    c->crec1 = k.take<float4>(N);
    c->cpos = k.take<float4>(N);
    c->csw = k.take<float4>(N);
    c->vrun_start = k.take<int>(N + 1);
    c->pose_R = k.take<float>(16);
    c->bsr = k.take<float>(nnzb * 144);
    c->grad = k.take<float>(P);
    c->pnode = k.take<float>(M * 72);
    c->minv = k.take<float>(M * 144);
    c->pose_blk = k.take<float>(72);
    c->dmom = k.take<float>(M * 72);
    c->bsr_s = k.take<float>(nnzb * 144);
    c->grad_s = k.take<float>(P);
    c->pnode_s = k.take<float>(M * 72);
    c->pblk_s = k.take<float>(36);
    c->x_prev = k.take<float>(M * 12);
    c->xm_prev = k.take<double>(M * 12);
    c->pose_prev = k.take<double>(6);
    c->node_energy = k.take<float2>(M);
    c->pix = k.take<int>(N);
    c->max_k1_ctas = (int)((N + ED_K1_THREADS - 1) / ED_K1_THREADS) + 1;
    c->k1_part = k.take<float2>((size_t)c->max_k1_ctas * ED_K1_PART);
    c->lb_ticket = k.take<unsigned long long>(1);
    c->lb_state = k.take<unsigned long long>((size_t)c->max_k1_ctas);
    c->vec_stride = (P + 63) / 64 * 64;
    c->vec = k.take<float>(6 * c->vec_stride);
    c->pcg_part = k.take<double>(2 * (size_t)ED_MAX_PCG_GRID * ED_PCG_PART);
    c->red_part = k.take<double>(4 * (size_t)ED_MAX_PCG_GRID);
    c->pcg_rows = k.take<int>(ED_MAX_PCG_GRID + 1);
    c->pcg_rows_b = k.take<int>(ED_MAX_PCG_GRID + 1);
    c->zbuf = k.take<unsigned long long>(WH);
    c->regpix = k.take<int>(WH);
    c->fused_pix = k.take<int>(N);
    c->flag_a = k.take<int>(big + 1);
    c->flag_b = k.take<int>(big + 1);
    c->scan_state_len = (int)((scan_len + 4095) / 4096 + 2);
    c->scan_state = k.take<unsigned long long>(c->scan_state_len);
    c->scan_ticket = k.take<unsigned>(64);
    c->gpts = k.take<float4>(2 * N);
    c->comb_pos = k.take<float4>(N);
    c->comb_nrm = k.take<float4>(N);
    return k.off + 256;
}

bool limits_ok(const ed_limits *L)
{
    return L && L->max_points > 0 && L->max_nodes >= 4 && L->max_nodes <= ED_HARD_MAX_NODES && L->max_width > 0 &&
           L->max_height > 0 && L->max_points < (1 << 27) && (long)L->max_width * L->max_height < (1L << 30);
}

}  // namespace

extern "C" ed_status ed_query_workspace(const ed_limits *limits, size_t *bytes)
{
    if (!limits_ok(limits) || !bytes) return ED_ERR_ARG;
    ed_context c;
    memset(&c, 0, sizeof(c));
    c.lim = *limits;
    normalise_limits(c.lim);
    *bytes = carve(&c, nullptr);
    return ED_OK;
}

extern "C" ed_status ed_create(const ed_limits *limits, void *workspace, size_t workspace_bytes, ed_context **out)
{
    if (!limits_ok(limits) || !workspace || !out || ((uintptr_t)workspace & 255)) return ED_ERR_ARG;
    ed_context *c = (ed_context *)calloc(1, sizeof(ed_context));
    if (!c) return ED_ERR_ARG;
    c->lim = *limits;
    normalise_limits(c->lim);
    size_t need = carve(c, nullptr);
    if (workspace_bytes < need) {
        free(c);
        return ED_ERR_CAPACITY;
    }
    carve(c, (char *)workspace);
    // pinned host buffers: the row pointer read back at graph build and the
    // staging of small host-to-device copies (no stream synchronisation)
    if (cudaMallocHost((void **)&c->row_ptr_host, sizeof(int) * ((size_t)c->lim.max_nodes + 1)) != cudaSuccess ||
        cudaMallocHost((void **)&c->pinned, sizeof(int) * ED_PINNED_INTS) != cudaSuccess) {
        if (c->row_ptr_host) cudaFreeHost(c->row_ptr_host);
        free(c);
        return ED_ERR_CUDA;
    }
    c->ws = (char *)workspace;
    c->ws_bytes = workspace_bytes;
    c->wait_ns = ED_BAR_TIMEOUT_NS;
    c->asm_pairs = 2;
    c->pt_chunk = 512;
    c->bar_extra = 0;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaMemset(c->misc, 0, sizeof(int) * MI_COUNT) != cudaSuccess ||
        cudaMemset(c->dmisc, 0, sizeof(double) * 64) != cudaSuccess ||
        cudaMemset(c->pcg_part, 0, sizeof(double) * 2 * (size_t)ED_MAX_PCG_GRID * ED_PCG_PART) != cudaSuccess ||
        cudaMemset(c->lb_ticket, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->lb_state, 0, sizeof(unsigned long long) * (size_t)c->max_k1_ctas) != cudaSuccess ||
        cudaMemset(c->scan_state, 0, sizeof(unsigned long long) * c->scan_state_len) != cudaSuccess ||
        cudaMemset(c->scan_ticket, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaFreeHost(c->row_ptr_host);
        cudaFreeHost(c->pinned);
        free(c);
        return ED_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_misc, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_build, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void **)&c->misc_host, sizeof(int) * MI_COUNT) != cudaSuccess) {
        if (c->aux) cudaStreamDestroy(c->aux);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        if (c->ev_misc) cudaEventDestroy(c->ev_misc);
        if (c->ev_build) cudaEventDestroy(c->ev_build);
        cudaFreeHost(c->row_ptr_host);
        cudaFreeHost(c->pinned);
        free(c);
        return ED_ERR_CUDA;
    }
    *out = c;
    return ED_OK;
}

extern "C" ed_status ed_destroy(ed_context *ctx)
{
    if (!ctx) return ED_ERR_ARG;
    if (ctx->build_pending) cudaEventSynchronize(ctx->ev_build);   // (its copies into pinned memory)
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_join);
    cudaEventDestroy(ctx->ev_misc);
    cudaEventDestroy(ctx->ev_build);
    cudaFreeHost(ctx->misc_host);
    cudaFreeHost(ctx->row_ptr_host);
    cudaFreeHost(ctx->pinned);
    free(ctx);
    return ED_OK;
}

extern "C" const char *ed_status_string(ed_status s)
{
    switch (s) {
    case ED_OK: return "ok";
    case ED_ERR_ARG: return "invalid argument";
    case ED_ERR_CUDA: return "CUDA error";
    case ED_ERR_CAPACITY: return "capacity exceeded";
    case ED_ERR_NONFINITE: return "non-finite value";
    case ED_ERR_BREAKDOWN: return "PCG breakdown";
    case ED_ERR_TIMEOUT: return "device wait timed out";
    case ED_ERR_STATE: return "invalid call order";
    }
    return "unknown status";
}

extern "C" ed_status ed_set_debug(ed_context *ctx, float *warped_pos, float *warped_nrm, int *pix)
{
    if (!ctx) return ED_ERR_ARG;
    ctx->dbg_wpos = warped_pos;
    ctx->dbg_wnrm = warped_nrm;
    ctx->dbg_pix = pix;
    return ED_OK;
}

static unsigned long long g_launches = 0;
void ed_note_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }
void ed_note_launches(unsigned long long n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }

extern "C" ed_status ed_set_keypoints(ed_context *ctx, const float *kp_pos, const float *kp_target, int n_keypoints,
                                      float w_corr)
{
    if (!ctx || n_keypoints < 0) return ED_ERR_ARG;
    if (n_keypoints > 0 && (!kp_pos || !kp_target || ((uintptr_t)kp_pos & 15) || ((uintptr_t)kp_target & 15) ||
                            !(w_corr >= 0.f)))
        return ED_ERR_ARG;
    ctx->kp_pos = n_keypoints > 0 ? (const float4 *)kp_pos : nullptr;
    ctx->kp_tgt = n_keypoints > 0 ? (const float4 *)kp_target : nullptr;
    ctx->n_kp = n_keypoints;
    ctx->w_corr = w_corr;
    ctx->have_graph = 0;   // the point set changes: build the graph again
    return ED_OK;
}

extern "C" ed_status ed_set_wait_limit(ed_context *ctx, unsigned long long limit_ns)
{
    if (!ctx) return ED_ERR_ARG;
    if (limit_ns == 0) limit_ns = ED_BAR_TIMEOUT_NS;
    if (limit_ns < ED_MIN_WAIT_NS) return ED_ERR_ARG;
    ctx->wait_ns = limit_ns;
    return ED_OK;
}

extern "C" ed_status ed_set_barrier_test(ed_context *ctx, int extra_arrivals)
{
    if (!ctx || extra_arrivals < 0 || extra_arrivals > 1024) return ED_ERR_ARG;
    ctx->bar_extra = extra_arrivals;
    return ED_OK;
}

extern "C" ed_status ed_launch_count(unsigned long long *count)
{
    if (!count) return ED_ERR_ARG;
    *count = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
    return ED_OK;
}

extern "C" ed_status ed_set_timing_every(ed_context *ctx, int kernel_id, cudaEvent_t *events, int n_pairs, int every,
                                        int *recorded)
{
    if (!ctx || n_pairs < 0 || (n_pairs > 0 && !events) || kernel_id < 0 || kernel_id > ED_KERNEL_GRAD || every < 1)
        return ED_ERR_ARG;
    ctx->tm_kernel = kernel_id;
    ctx->tm_events = n_pairs > 0 ? events : nullptr;
    ctx->tm_pairs = n_pairs;
    ctx->tm_count = 0;
    ctx->tm_every = every;
    ctx->tm_seen = 0;
    ctx->tm_recorded = recorded;
    if (recorded) *recorded = 0;
    return ED_OK;
}

extern "C" ed_status ed_set_timing(ed_context *ctx, int kernel_id, cudaEvent_t *events, int n_pairs, int *recorded)
{
    return ed_set_timing_every(ctx, kernel_id, events, n_pairs, 1, recorded);
}

extern "C" ed_status ed_graph_info(ed_context *ctx, int *m, int *nnzb, int *n_entries, int *n_runs)
{
    if (!ctx) return ED_ERR_ARG;
    if (!ctx->have_graph) return ED_ERR_STATE;
    if (nnzb || n_entries || n_runs) {   // the pattern's counts: the build's queued work must have reached them
        ed_status s = ed_graph_ready(ctx, 0);
        if (s != ED_OK) return s;
        ED_CUDA_TRY(cudaStreamSynchronize(0));   // (the plan's copy on the legacy stream)
    }
    if (m) *m = ctx->m;
    if (nnzb) *nnzb = ctx->nnzb;
    if (n_entries) *n_entries = ctx->n_entries;
    if (n_runs) *n_runs = ctx->n_runs;
    return ED_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan of int arrays (out[n] = total) in one pass: decoupled
// look-back over tiles of 4096.  Tiles take increasing ticket numbers in the
// order CTAs start, so a tile only waits for tiles that are already running.
// Every tile publishes its aggregate, then its inclusive prefix, as one 64-bit
// word tagged with the scan's epoch (words of older scans never match); the
// wait for a predecessor gives up after the context's wait limit (ED_ERR_TIMEOUT).
// ---------------------------------------------------------------------------

#define DS_T 256
#define DS_PER 16
#define DS_TILE (DS_T * DS_PER)
#define DS_AGG 1u
#define DS_INC 2u

__device__ __forceinline__ unsigned long long ds_load(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void ds_store(unsigned long long *p, unsigned epoch, unsigned flag, int v)
{
    const unsigned long long w = ((unsigned long long)((epoch << 2) | flag) << 32) | (unsigned)v;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__global__ void __launch_bounds__(DS_T) k_scan_dlb(const int *in, int *out, int n, const int *n_dev, int *total2,
                                                   unsigned long long *state, unsigned *ticket, unsigned ticket_base,
                                                   unsigned epoch, int *status, unsigned long long wait_ns)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ int s_tile, s_excl, s_warp[DS_T / 32];
    if (threadIdx.x == 0) s_tile = (int)(atomicAdd(ticket, 1u) - ticket_base);
    __syncthreads();
    const int tile = s_tile;
    if (n_dev) {   // the length read on the device (n: the launch's capacity); later tiles only take a ticket
        const int nd = *n_dev;
        n = nd <= n ? nd : 0;   // (a length above the capacity is an error reported elsewhere: nothing scanned)
        if (n <= 0) {
            if (tile == 0 && threadIdx.x == 0) {
                out[0] = 0;
                if (total2) *total2 = 0;
            }
            return;
        }
        if ((long)tile * DS_TILE >= n) return;
    }
    const long base = (long)tile * DS_TILE + (long)threadIdx.x * DS_PER;
    int v[DS_PER], sum = 0;
    if (base + DS_PER <= n && !((uintptr_t)(in + base) & 15)) {
        const int4 *p4 = reinterpret_cast<const int4 *>(in + base);
#pragma unroll
        for (int q = 0; q < DS_PER / 4; ++q) {
            const int4 w = p4[q];
            v[4 * q] = w.x;
            v[4 * q + 1] = w.y;
            v[4 * q + 2] = w.z;
            v[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < DS_PER; ++e) v[e] = base + e < n ? in[base + e] : 0;
    }
#pragma unroll
    for (int e = 0; e < DS_PER; ++e) sum += v[e];
    // exclusive prefix of the thread sums within the tile
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < DS_T / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < DS_T / 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < DS_T / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const int aggregate = s_warp[DS_T / 32 - 1];
    int run = (wid > 0 ? s_warp[wid - 1] : 0) + x - sum;
    // the tile's exclusive prefix from its predecessors
    if (threadIdx.x == 0) {
        int excl = 0;
        if (tile == 0) {
            ds_store(state, epoch, DS_INC, aggregate);
        } else {
            ds_store(state + tile, epoch, DS_AGG, aggregate);
            const unsigned long long t0 = ed_gtimer();
            unsigned spins = 0;
            for (int p = tile - 1; p >= 0;) {
                const unsigned long long w = ds_load(state + p);
                const unsigned hi = (unsigned)(w >> 32), fl = hi & 3u;
                if ((hi >> 2) != epoch || fl == 0u) {
                    if ((++spins & 63u) == 0 && ed_gtimer() - t0 > wait_ns) {
                        atomicCAS(status, ED_OK, ED_ERR_TIMEOUT);
                        break;
                    }
                    continue;
                }
                excl += (int)(unsigned)w;
                if (fl == DS_INC) break;
                --p;
            }
            ds_store(state + tile, epoch, DS_INC, excl + aggregate);
        }
        s_excl = excl;
    }
    __syncthreads();
    run += s_excl;
#pragma unroll
    for (int e = 0; e < DS_PER; ++e) {
        if (base + e < n) out[base + e] = run;
        run += v[e];
        if (base + e == n - 1) {
            out[n] = run;
            if (total2) *total2 = run;
        }
    }
}

__global__ void k_set_zero_at(int *p, int *p2)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    *p = 0;
    if (p2) *p2 = 0;
}

ed_status ed_scan_exclusive(ed_context *ctx, const int *in, int *out, int n, cudaStream_t st, int *total2,
                            const int *n_dev)
{
    if (n <= 0) {
        ED_LAUNCH(k_set_zero_at, 1, 1, st, out, total2); ed_note_launch();
        ED_LAUNCH_CHECK();
        return ED_OK;
    }
    const int tiles = ed_div_up(n, DS_TILE);
    if (tiles > ctx->scan_state_len) return ED_ERR_CAPACITY;
    unsigned epoch = ++ctx->scan_epoch;
    if (epoch >= (1u << 30)) {   // epochs wrap: clear the words of old scans
        ED_CUDA_TRY(cudaMemsetAsync(ctx->scan_state, 0, sizeof(unsigned long long) * ctx->scan_state_len, st));
        ctx->scan_epoch = epoch = 1;
    }
    ED_LAUNCH(k_scan_dlb, tiles, DS_T, st, in, out, n, n_dev, total2, ctx->scan_state, ctx->scan_ticket, ctx->scan_ticket_base, epoch,
                                       ctx->misc + MI_STATUS, ctx->wait_ns); ed_note_launch();
    ctx->scan_ticket_base += (unsigned)tiles;
    ED_LAUNCH_CHECK();
    return ED_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, value) pairs, 8 bits per pass
// ---------------------------------------------------------------------------

#define RX_TILE 1024

__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int n, int shift, int ntiles, int *__restrict__ cnt)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long base = (long)blockIdx.x * RX_TILE;
    for (int e = threadIdx.x; e < RX_TILE; e += 256)
        if (base + e < n) atomicAdd(&h[(keys[base + e] >> shift) & 255u], 1);
    __syncthreads();
    cnt[(long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// one warp per tile; the tile's keys and values are loaded up front (32 per
// lane, one round of loads), then visited in order, 32 at a time; equal digits
// keep their order
__global__ void __launch_bounds__(32) k_radix_scatter(const uint32_t *__restrict__ keys,
                                                      const uint32_t *__restrict__ vals, int n, int shift, int ntiles,
                                                      const int *__restrict__ offs, uint32_t *__restrict__ ko,
                                                      uint32_t *__restrict__ vo)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ int c[256];
    const int tile = blockIdx.x;
    const int lane = threadIdx.x;
    const long base = (long)tile * RX_TILE;
    uint32_t kk[RX_TILE / 32], vv[RX_TILE / 32];
#pragma unroll
    for (int r = 0; r < RX_TILE / 32; ++r) {
        const long e = base + 32 * r + lane;
        kk[r] = e < n ? keys[e] : 0u;
        vv[r] = e < n ? vals[e] : 0u;
    }
    for (int d = lane; d < 256; d += 32) c[d] = offs[(long)d * ntiles + tile];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RX_TILE / 32; ++r) {
        const long e = base + 32 * r + lane;
        const bool ok = e < n;
        const uint32_t k = kk[r];
        const int d = ok ? (int)((k >> shift) & 255u) : 256 + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        const int pos = ok ? c[d] + rank : 0;
        __syncwarp();
        if (ok && rank == 0) c[d] += __popc(peers);
        __syncwarp();
        if (ok) {
            ko[pos] = k;
            vo[pos] = vv[r];
        }
    }
}

ed_status ed_radix_sort_pairs(ed_context *ctx, uint32_t *keys, uint32_t *vals, int n, int key_bits, cudaStream_t st)
{
    if (n <= 1) return ED_OK;
    const int ntiles = ed_div_up(n, RX_TILE);
    uint32_t *ka = keys, *va = vals, *kb = ctx->ent_key2, *vb = ctx->ent_val2;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        ED_LAUNCH(k_radix_hist, ntiles, 256, st, ka, n, shift, ntiles, ctx->radix_cnt); ed_note_launch();
        ED_LAUNCH_CHECK();
        ed_status s = ed_scan_exclusive(ctx, ctx->radix_cnt, ctx->radix_cnt, 256 * ntiles, st);
        if (s != ED_OK) return s;
        ED_LAUNCH(k_radix_scatter, ntiles, 32, st, ka, va, n, shift, ntiles, ctx->radix_cnt, kb, vb); ed_note_launch();
        ED_LAUNCH_CHECK();
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
        passes++;
    }
    if (ka != keys) {
        ED_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
        ED_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return ED_OK;
}

// ---------------------------------------------------------------------------
// target normal map (data term n(u), Sec. II.E)
// ---------------------------------------------------------------------------

__global__ void k_normals(const float *__restrict__ depth, ed_intrinsics K, int h, float4 *__restrict__ nmap)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= K.width || v >= K.height) return;
    const int W = K.width;
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (u - h >= 0 && u + h < W && v - h >= 0 && v + h < K.height) {
        const float Dc = __ldg(depth + v * W + u);
        const float Dl = __ldg(depth + v * W + u - h), Dr = __ldg(depth + v * W + u + h);
        const float Du = __ldg(depth + (v - h) * W + u), Dd = __ldg(depth + (v + h) * W + u);
        if (Dc > 0.f && Dl > 0.f && Dr > 0.f && Du > 0.f && Dd > 0.f) {
            const float ifx = 1.0f / K.fx, ify = 1.0f / K.fy;
            const float xl = ((float)(u - h) - K.cx) * Dl * ifx, yl = ((float)v - K.cy) * Dl * ify;
            const float xr = ((float)(u + h) - K.cx) * Dr * ifx, yr = ((float)v - K.cy) * Dr * ify;
            const float xu = ((float)u - K.cx) * Du * ifx, yu = ((float)(v - h) - K.cy) * Du * ify;
            const float xd = ((float)u - K.cx) * Dd * ifx, yd = ((float)(v + h) - K.cy) * Dd * ify;
            const float ax = xd - xu, ay = yd - yu, az = Dd - Du;   // V(u, v+h) - V(u, v-h)
            const float bx = xr - xl, by = yr - yl, bz = Dr - Dl;   // V(u+h, v) - V(u-h, v)
            float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
            const float l2 = nx * nx + ny * ny + nz * nz;
            if (l2 > 0.f) {
                float s = rsqrtf(l2);
                if (nz > 0.f) s = -s;
                o = make_float4(nx * s, ny * s, nz * s, 1.0f);
            }
        }
    }
    nmap[v * W + u] = o;
}

extern "C" ed_status ed_compute_normals(ed_context *ctx, const float *depth, ed_intrinsics intr, int half_width,
                                        float *nmap, cudaStream_t stream)
{
    if (!ctx || !depth || !nmap || intr.width <= 0 || intr.height <= 0 || half_width < 1 ||
        !(intr.fx > 0.f) || !(intr.fy > 0.f) || ((uintptr_t)nmap & 15))
        return ED_ERR_ARG;
    dim3 b(32, 8), g(ed_div_up(intr.width, 32), ed_div_up(intr.height, 8));
    ED_LAUNCH(k_normals, g, b, stream, depth, intr, half_width, (float4 *)nmap); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}

// ---------------------------------------------------------------------------
// Eq. (1) warp of a point set
// ---------------------------------------------------------------------------

__global__ void k_warp(const float4 *__restrict__ pos, const float4 *__restrict__ nrm, const ushort4 *__restrict__ idx,
                       const float4 *__restrict__ w, const float4 *__restrict__ g, const float4 *__restrict__ x4,
                       const double *__restrict__ pose, int n, float4 *__restrict__ pos_out, float4 *__restrict__ nrm_out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ ed_pose_f P;
    if (threadIdx.x == 0) ed_pose_eval(pose, P);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos[i], nr = nrm[i];
    ed_warped W = ed_warp_point(p, nr, idx[i], w[i], g, x4, P.R, P.T);
    pos_out[i] = make_float4(W.v.x, W.v.y, W.v.z, p.w);
    nrm_out[i] = make_float4(W.n.x, W.n.y, W.n.z, nr.w);
}

struct ResetPose {
    double v[6];
};

// identity warp (A_j = I, t_j = 0) for the first m nodes, the FP64 master copy
// likewise, the pose from its prior
__global__ void k_reset_params(int m, float *__restrict__ x, double *__restrict__ xm, double *__restrict__ pose,
                               ResetPose prior)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 12 * m) {
        const int e = i % 12;
        const float v = (e == 0 || e == 5 || e == 10) ? 1.0f : 0.0f;
        x[i] = v;
        if (xm) xm[i] = (double)v;
    } else if (i < 12 * m + 6) {
        pose[i - 12 * m] = prior.v[i - 12 * m];
    }
}

extern "C" ed_status ed_reset_params(ed_context *ctx, float *x, double *x_master, double *pose,
                                     const double *prior_host, cudaStream_t st)
{
    if (!ctx || !x || !pose) return ED_ERR_ARG;
    if (!ctx->have_graph) return ED_ERR_STATE;
    ResetPose pr;
    for (int k = 0; k < 6; ++k) pr.v[k] = prior_host ? prior_host[k] : 0.0;
    const int m = ctx->m;
    ED_LAUNCH(k_reset_params, ed_div_up(12 * m + 6, 256), 256, st, m, x, x_master, pose, pr); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}

extern "C" ed_status ed_warp(ed_context *ctx, const float *x, const double *pose, const float *pos_in,
                             const float *nrm_in, int n_points, float *pos_out, float *nrm_out, cudaStream_t stream)
{
    if (!ctx || !x || !pose || !pos_in || !nrm_in || !pos_out || !nrm_out || n_points < 0) return ED_ERR_ARG;
    if (!ctx->have_graph) return ED_ERR_STATE;
    if (n_points > ctx->N) return ED_ERR_ARG;   // the skinning of the graph covers the model points
    if (n_points == 0) return ED_OK;
    ED_LAUNCH(k_warp, ed_div_up(n_points, 256), 256, stream, 
        (const float4 *)pos_in, (const float4 *)nrm_in, (const ushort4 *)ctx->graph.idx,
        (const float4 *)ctx->graph.weights, (const float4 *)ctx->graph.nodes, (const float4 *)x, pose, n_points,
        (float4 *)pos_out, (float4 *)nrm_out); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}
