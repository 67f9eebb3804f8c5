// graph.cu -- ed_build_graph: ED nodes, nearest nodes and weights, node
// graph, and the block structure of the normal equations (Sec. II.D-II.E).
#include <math.h>
#include <string.h>

#include "ed_internal.cuh"

// ordered-int image of a float (monotone for signed comparison)
__device__ __forceinline__ int f2o(float f)
{
    int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

__global__ void k_bbox_init(int *misc)
{
    if (threadIdx.x < 3) {
        misc[MI_BBOX + threadIdx.x] = 0x7fffffff;
        misc[MI_BBOX + 3 + threadIdx.x] = (int)0x80000000;
    }
}

__global__ void k_bbox(const float4 *__restrict__ pos, int n, int *misc)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 p = pos[i];
        mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; ++d) {
            atomicMin(&misc[MI_BBOX + d], f2o(mn[d]));
            atomicMax(&misc[MI_BBOX + 3 + d], f2o(mx[d]));
        }
}

// cell size, inverse and dims of the sampling grid (edge r / sqrt 3) and of the
// search grid (edge kc), by the same FP32 operations as the oracle
__global__ void k_grid_setup(int *misc, float *fmisc, float r, float kc, long max_cells, int sampling)
{
    float mn[3], mx[3];
    for (int d = 0; d < 3; ++d) {
        mn[d] = o2f(misc[MI_BBOX + d]);
        mx[d] = o2f(misc[MI_BBOX + 3 + d]);
        fmisc[MF_BBOX + d] = mn[d];
        fmisc[MF_BBOX + 3 + d] = mx[d];
    }
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 0 && !sampling) {
            misc[MI_DIMS + 3] = 0;
            continue;
        }
        float cs = pass == 0 ? __fmul_rn(r, 0.577350269f) : kc;
        float inv = __fdiv_rn(1.0f, cs);
        long cells = 1;
        int dims[3];
        for (int d = 0; d < 3; ++d) {
            float t = __fmul_rn(__fsub_rn(mx[d], mn[d]), inv);
            dims[d] = (int)floorf(t) + 1;
            cells *= dims[d];
        }
        const int base = pass == 0 ? MI_DIMS : MI_KDIMS;
        if (cells > max_cells || cells <= 0 || !(cs > 0.f)) {
            misc[MI_STATUS] = ED_ERR_CAPACITY;
            cells = 0;
        }
        for (int d = 0; d < 3; ++d) misc[base + d] = dims[d];
        misc[base + 3] = (int)cells;
        fmisc[pass == 0 ? MF_CELL : MF_KCELL] = cs;
        fmisc[pass == 0 ? MF_INV : MF_KINV] = inv;
    }
    fmisc[MF_R2] = __fmul_rn(r, r);
}

__device__ __forceinline__ int3 cell3(float x, float y, float z, const float *fmisc, float inv, const int *dims)
{
    int c[3];
    const float p[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float t = __fmul_rn(__fsub_rn(p[d], fmisc[MF_BBOX + d]), inv);
        int ci = (int)floorf(t);
        ci = ci < 0 ? 0 : (ci >= dims[d] ? dims[d] - 1 : ci);
        c[d] = ci;
    }
    return make_int3(c[0], c[1], c[2]);
}

__global__ void k_cell_of(const float4 *__restrict__ pos, int n, const int *__restrict__ misc,
                          const float *__restrict__ fmisc, int *__restrict__ cell_of)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int dims[3] = {misc[MI_DIMS], misc[MI_DIMS + 1], misc[MI_DIMS + 2]};
    const float4 p = pos[i];
    int3 c = cell3(p.x, p.y, p.z, fmisc, fmisc[MF_INV], dims);
    cell_of[i] = c.x + dims[0] * (c.y + dims[1] * c.z);
}

// Poisson-disk phase, step 1: every point of a cell of this phase that keeps
// distance >= r (FP32 key) from all nodes chosen so far bids for its cell; the
// lowest index wins.  Nodes within r lie in the 5x5x5 cells around the point.
__global__ void k_poisson_pick(const float4 *__restrict__ pos, int n, int phase, const int *__restrict__ misc,
                               const float *__restrict__ fmisc, const int *__restrict__ cell_of,
                               const int *__restrict__ cell_node, int *__restrict__ cell_pick)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nx = misc[MI_DIMS], ny = misc[MI_DIMS + 1], nz = misc[MI_DIMS + 2];
    const int c = cell_of[i];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    if ((cx % 3) + 3 * (cy % 3) + 9 * (cz % 3) != phase) return;
    const float4 p = pos[i];
    const float r2 = fmisc[MF_R2];
    for (int dz = -2; dz <= 2; ++dz) {
        const int az = cz + dz;
        if (az < 0 || az >= nz) continue;
        for (int dy = -2; dy <= 2; ++dy) {
            const int ay = cy + dy;
            if (ay < 0 || ay >= ny) continue;
            for (int dx = -2; dx <= 2; ++dx) {
                const int ax = cx + dx;
                if (ax < 0 || ax >= nx) continue;
                const int q = cell_node[ax + nx * (ay + ny * az)];
                if (q < 0) continue;
                const float4 g = pos[q];
                if (ed_key(p.x, p.y, p.z, g.x, g.y, g.z) < r2) return;
            }
        }
    }
    atomicMin(&cell_pick[c], i);
}

// Poisson-disk phase, step 2 (one CTA): the phase's cells in increasing linear
// order receive consecutive node numbers
__global__ void k_poisson_commit(const float4 *__restrict__ pos, int phase, int *__restrict__ misc,
                                 const int *__restrict__ cell_pick, int *__restrict__ cell_node, float4 *__restrict__ nodes,
                                 int max_nodes)
{
    __shared__ int sh[33];
    __shared__ int base_s;
    const int nx = misc[MI_DIMS], ny = misc[MI_DIMS + 1], nz = misc[MI_DIMS + 2];
    const int px = phase % 3, py = (phase / 3) % 3, pz = phase / 9;
    const int ax = nx > px ? (nx - px + 2) / 3 : 0, ay = ny > py ? (ny - py + 2) / 3 : 0,
              az = nz > pz ? (nz - pz + 2) / 3 : 0;
    const long total = (long)ax * ay * az;
    if (threadIdx.x == 0) base_s = misc[MI_PHASE_BASE];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long t0 = 0; t0 < total; t0 += blockDim.x) {
        const long t = t0 + threadIdx.x;
        int L = -1, pick = -1;
        if (t < total) {
            const int a = (int)(t % ax), b = (int)((t / ax) % ay), c = (int)(t / ((long)ax * ay));
            L = (px + 3 * a) + nx * ((py + 3 * b) + ny * (pz + 3 * c));
            const int pk = cell_pick[L];
            if (pk != 0x7f7f7f7f) pick = pk;   // 0x7f7f7f7f: no bid (memset pattern)
        }
        const int f = pick >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int wpre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) sh[wid] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < nw; ++w) {
                int v = sh[w];
                sh[w] = s;
                s += v;
            }
            sh[32] = s;
        }
        __syncthreads();
        if (f) {
            const int id = base_s + sh[wid] + wpre;
            cell_node[L] = pick;
            if (id < max_nodes) {
                const float4 p = pos[pick];
                nodes[id] = make_float4(p.x, p.y, p.z, 0.f);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += sh[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) misc[MI_PHASE_BASE] = base_s;
}

// ---------------------------------------------------------------------------
// nearest-node search grid
// ---------------------------------------------------------------------------

__global__ void k_kcell_count(const float4 *__restrict__ nodes, int m, const int *__restrict__ misc,
                              const float *__restrict__ fmisc, int *__restrict__ cnt, int *__restrict__ cell_of_node)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int dims[3] = {misc[MI_KDIMS], misc[MI_KDIMS + 1], misc[MI_KDIMS + 2]};
    const float4 g = nodes[j];
    int3 c = cell3(g.x, g.y, g.z, fmisc, fmisc[MF_KINV], dims);
    const int L = c.x + dims[0] * (c.y + dims[1] * c.z);
    cell_of_node[j] = L;
    atomicAdd(&cnt[L], 1);
}

__global__ void k_kcell_fill(int m, const int *__restrict__ start, int *__restrict__ fill,
                             const int *__restrict__ cell_of_node, int *__restrict__ kn)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int L = cell_of_node[j];
    kn[start[L] + atomicAdd(&fill[L], 1)] = j;
}

#define KNN_S 5   // K + 1 nearest (Eq. 2 needs the (K+1)-th distance)

__device__ __forceinline__ void topk_ins(float *kk, int *ii, float key, int id)
{
    if (key > kk[KNN_S - 1] || (key == kk[KNN_S - 1] && id >= ii[KNN_S - 1])) return;
    int p = KNN_S - 1;
    while (p > 0 && (kk[p - 1] > key || (kk[p - 1] == key && ii[p - 1] > id))) {
        kk[p] = kk[p - 1];
        ii[p] = ii[p - 1];
        --p;
    }
    kk[p] = key;
    ii[p] = id;
}

// K+1 nearest nodes by rings of search cells; a ring R is the last one needed
// once the (K+1)-th key is below (R * cell)^2 (with a round-off margin): every
// node outside rings 0..R is at least R cells away.  Then the weights.
__global__ void k_knn(const float4 *__restrict__ pos, int n, const float4 *__restrict__ nodes, int m,
                      const int *__restrict__ misc, const float *__restrict__ fmisc, const int *__restrict__ start,
                      const int *__restrict__ kn, int mode, float sigma, ushort4 *__restrict__ idx_out,
                      float4 *__restrict__ w_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int dims[3] = {misc[MI_KDIMS], misc[MI_KDIMS + 1], misc[MI_KDIMS + 2]};
    const float kc = fmisc[MF_KCELL];
    const float4 p = pos[i];
    const int3 c = cell3(p.x, p.y, p.z, fmisc, fmisc[MF_KINV], dims);
    float kk[KNN_S];
    int ii[KNN_S];
#pragma unroll
    for (int s = 0; s < KNN_S; ++s) {
        kk[s] = INFINITY;
        ii[s] = 0x7fffffff;
    }
    const int need = m < KNN_S ? m : KNN_S;
    int maxR = dims[0];
    if (dims[1] > maxR) maxR = dims[1];
    if (dims[2] > maxR) maxR = dims[2];
    for (int R = 0; R <= maxR; ++R) {
        for (int dz = -R; dz <= R; ++dz) {
            const int az = c.z + dz;
            if (az < 0 || az >= dims[2]) continue;
            for (int dy = -R; dy <= R; ++dy) {
                const int ay = c.y + dy;
                if (ay < 0 || ay >= dims[1]) continue;
                const bool edge_yz = (dz == -R || dz == R || dy == -R || dy == R);
                for (int dx = -R; dx <= R; dx += (edge_yz ? 1 : 2 * (R > 0 ? R : 1))) {
                    const int ax = c.x + dx;
                    if (ax >= 0 && ax < dims[0]) {
                        const int L = ax + dims[0] * (ay + dims[1] * az);
                        for (int t = start[L]; t < start[L + 1]; ++t) {
                            const int j = kn[t];
                            const float4 g = __ldg(nodes + j);
                            topk_ins(kk, ii, ed_key(p.x, p.y, p.z, g.x, g.y, g.z), j);
                        }
                    }
                    if (R == 0) break;
                }
            }
        }
        if (need > 0 && kk[need - 1] < INFINITY) {
            const float b = (float)R * kc;
            if (kk[need - 1] < b * b * 0.99999f) break;
        }
    }
    // weights (Eq. 1 normalised; Gaussian or Eq. 2)
    float w[4], sum = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float t;
        if (ii[s] == 0x7fffffff) t = 0.f;
        else if (mode == ED_WEIGHT_GAUSSIAN) t = expf(-kk[s] / (2.0f * sigma * sigma));
        else {
            const float dmax = sqrtf(kk[4]);
            t = dmax > 0.f ? 1.0f - sqrtf(kk[s]) / dmax : 1.0f;
        }
        if (!(t > 0.f)) t = 0.f;
        w[s] = t;
        sum += t;
    }
    const float inv = sum > 0.f ? 1.0f / sum : 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) w[s] = sum > 0.f ? w[s] * inv : 0.25f;
    unsigned short id4[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) id4[s] = (unsigned short)(ii[s] == 0x7fffffff ? 0 : ii[s]);
    idx_out[i] = make_ushort4(id4[0], id4[1], id4[2], id4[3]);
    w_out[i] = make_float4(w[0], w[1], w[2], w[3]);
}

// N(j): the k_graph nearest other nodes (brute force over all nodes)
__global__ void k_node_graph(const float4 *__restrict__ nodes, int m, int kg, int *__restrict__ nbr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float kk[ED_MAX_KG];
    int ii[ED_MAX_KG];
    for (int s = 0; s < kg; ++s) {
        kk[s] = INFINITY;
        ii[s] = 0x7fffffff;
    }
    const float4 g = nodes[j];
    for (int l = 0; l < m; ++l) {
        if (l == j) continue;
        const float4 h = __ldg(nodes + l);
        const float key = ed_key(g.x, g.y, g.z, h.x, h.y, h.z);
        if (key > kk[kg - 1] || (key == kk[kg - 1] && l >= ii[kg - 1])) continue;
        int p = kg - 1;
        while (p > 0 && (kk[p - 1] > key || (kk[p - 1] == key && ii[p - 1] > l))) {
            kk[p] = kk[p - 1];
            ii[p] = ii[p - 1];
            --p;
        }
        kk[p] = key;
        ii[p] = l;
    }
    for (int s = 0; s < kg; ++s) nbr[j * kg + s] = ii[s] == 0x7fffffff ? -1 : ii[s];
}

// ---------------------------------------------------------------------------
// block pattern of J^T J: node pairs sharing a point, node-graph edges, diagonal
// ---------------------------------------------------------------------------

__device__ __forceinline__ void set_bit(uint32_t *bm, int words, int a, int b)
{
    uint32_t *w = bm + (long)a * words + (b >> 5);
    const uint32_t bit = 1u << (b & 31);
    if (!(*w & bit)) atomicOr(w, bit);
}

__global__ void k_pairs_points(const ushort4 *__restrict__ idx, int n, uint32_t *bm, int words)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ushort4 q = idx[i];
    const int id[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (a != b) set_bit(bm, words, id[a], id[b]);
}

__global__ void k_pairs_graph(const int *__restrict__ nbr, int m, int kg, uint32_t *bm, int words)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    set_bit(bm, words, j, j);
    for (int s = 0; s < kg; ++s) {
        const int k = nbr[j * kg + s];
        if (k < 0) continue;
        set_bit(bm, words, j, k);
        set_bit(bm, words, k, j);
    }
}

__global__ void k_row_count(const uint32_t *__restrict__ bm, int m, int words, int *__restrict__ cnt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int c = 0;
    for (int w = 0; w < words; ++w) c += __popc(bm[(long)j * words + w]);
    cnt[j] = c;
}

__global__ void k_row_fill(const uint32_t *__restrict__ bm, int m, int words, const int *__restrict__ row_ptr,
                           int *__restrict__ col, int *__restrict__ brow, int *__restrict__ diag_pos)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int p = row_ptr[j];
    for (int w = 0; w < words; ++w) {
        uint32_t v = bm[(long)j * words + w];
        while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1;
            const int l = (w << 5) + b;
            if (l == j) diag_pos[j] = p;
            col[p] = l;
            brow[p] = j;
            ++p;
        }
    }
}

__device__ __forceinline__ int find_block(const int *__restrict__ row_ptr, const int *__restrict__ col, int j, int l)
{
    int lo = row_ptr[j], hi = row_ptr[j + 1] - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int c = col[mid];
        if (c == l) return mid;
        if (c < l) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void k_tpos(int nnzb, const int *__restrict__ row_ptr, const int *__restrict__ col,
                       const int *__restrict__ brow, int *__restrict__ tpos, int *__restrict__ upper_flag)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnzb) return;
    const int j = brow[b], l = col[b];
    tpos[b] = find_block(row_ptr, col, l, j);
    upper_flag[b] = l >= j;
}

__global__ void k_compact_upper(int nnzb, const int *__restrict__ flag, const int *__restrict__ pre,
                                int *__restrict__ up_list)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnzb) return;
    if (flag[b]) up_list[pre[b]] = b;
}

// one entry per (point, unordered slot pair s <= t): key = upper block, value =
// point << 4 | row slot << 2 | column slot, generated in point order
__global__ void k_entries_gen(const ushort4 *__restrict__ idx, int n, const int *__restrict__ row_ptr,
                              const int *__restrict__ col, uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                              int *__restrict__ status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ushort4 q = idx[i];
    const int id[4] = {q.x, q.y, q.z, q.w};
    int e = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = s; t < 4; ++t) {
            int j = id[s], l = id[t], sr = s, sc = t;
            if (j > l) {
                j = id[t];
                l = id[s];
                sr = t;
                sc = s;
            }
            const int b = find_block(row_ptr, col, j, l);
            if (b < 0) atomicExch(status, ED_ERR_STATE);
            key[10L * i + e] = (uint32_t)(b < 0 ? 0 : b);
            val[10L * i + e] = ((uint32_t)i << 4) | ((uint32_t)sr << 2) | (uint32_t)sc;
            ++e;
        }
}

__global__ void k_ent_count(const uint32_t *__restrict__ key, int ne, int *__restrict__ cnt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) atomicAdd(&cnt[key[e]], 1);
}

__global__ void k_chunk_count(int nnzb, const int *__restrict__ cnt, const int *__restrict__ brow,
                              const int *__restrict__ col, int *__restrict__ ccnt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnzb) return;
    const int c = (cnt[b] + ED_CHUNK - 1) / ED_CHUNK;
    ccnt[b] = brow[b] == col[b] ? 2 * c : (col[b] > brow[b] ? c : 0);
}

__global__ void k_chunk_fill(int nnzb, const int *__restrict__ cnt, const int *__restrict__ ent_start,
                             const int *__restrict__ brow, const int *__restrict__ col,
                             const int *__restrict__ cstart, int4 *__restrict__ chunks)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnzb || col[b] < brow[b]) return;
    const int n = cnt[b];
    const int per = (n + ED_CHUNK - 1) / ED_CHUNK;
    const int roles = brow[b] == col[b] ? 2 : 1;
    int q = cstart[b];
    for (int r = 0; r < roles; ++r)
        for (int k = 0; k < per; ++k) {
            const int beg = ent_start[b] + k * ED_CHUNK;
            const int c = min(ED_CHUNK, n - k * ED_CHUNK);
            chunks[q++] = make_int4(b, beg, c, r);
        }
}

// ---------------------------------------------------------------------------

static ed_status read_misc(ed_context *ctx, int *host, cudaStream_t st)
{
    ED_CUDA_TRY(cudaMemcpyAsync(host, ctx->misc, sizeof(int) * MI_COUNT, cudaMemcpyDeviceToHost, st));
    ED_CUDA_TRY(cudaStreamSynchronize(st));
    return ED_OK;
}

extern "C" ed_status ed_build_graph(ed_context *ctx, const float *pos, const float *nrm, int n_points, int m_in,
                                    const ed_graph_params *prm, const ed_graph *graph, cudaStream_t st)
{
    if (!ctx || !pos || !nrm || !prm || !graph || !graph->nodes || !graph->idx || !graph->weights || !graph->nbr ||
        !graph->counts)
        return ED_ERR_ARG;
    if (n_points <= 0 || n_points > ctx->lim.max_points || prm->k != ED_K || prm->k_graph < 1 ||
        prm->k_graph > ED_MAX_KG || m_in < 0 || m_in > ctx->lim.max_nodes)
        return ED_ERR_ARG;
    if (((uintptr_t)pos & 15) || ((uintptr_t)nrm & 15) || ((uintptr_t)graph->nodes & 15) ||
        ((uintptr_t)graph->weights & 15) || ((uintptr_t)graph->idx & 7))
        return ED_ERR_ARG;
    if (prm->weight_mode == ED_WEIGHT_GAUSSIAN && !(prm->sigma > 0.f)) return ED_ERR_ARG;
    const int max_nodes = m_in > 0 ? m_in : prm->max_nodes;
    if (m_in == 0 && (!(prm->node_radius > 0.f) || max_nodes <= 0 || max_nodes > ctx->lim.max_nodes)) return ED_ERR_ARG;

    ctx->have_graph = 0;
    ctx->have_system = 0;
    ctx->have_energy = 0;
    const int N = n_points;
    const float4 *P4 = (const float4 *)pos;
    float4 *G4 = (float4 *)graph->nodes;
    int hm[MI_COUNT];
    ed_status s;
    ED_CUDA_TRY(cudaMemsetAsync(ctx->misc, 0, sizeof(int) * MI_COUNT, st));

    // ---- bounding box and grids ----
    k_bbox_init<<<1, 32, 0, st>>>(ctx->misc); ed_note_launch();
    k_bbox<<<min(ed_div_up(N, 256), 4 * ctx->num_sms), 256, 0, st>>>(P4, N, ctx->misc); ed_note_launch();
    float kc = prm->search_cell;
    if (!(kc > 0.f)) kc = m_in > 0 ? (prm->sigma > 0.f ? prm->sigma : 1.0f) : 2.0f * prm->node_radius;
    k_grid_setup<<<1, 1, 0, st>>>(ctx->misc, ctx->fmisc, m_in > 0 ? 1.0f : prm->node_radius, kc, ctx->lim.max_cells,
                                  m_in == 0); ed_note_launch();
    ED_LAUNCH_CHECK();
    if ((s = read_misc(ctx, hm, st)) != ED_OK) return s;
    if (hm[MI_STATUS] != ED_OK) return (ed_status)hm[MI_STATUS];

    // ---- nodes ----
    int m;
    if (m_in == 0) {
        const int cells = hm[MI_DIMS + 3];
        ED_CUDA_TRY(cudaMemsetAsync(ctx->cell_pick, 0x7f, sizeof(int) * cells, st));
        ED_CUDA_TRY(cudaMemsetAsync(ctx->cell_node, 0xff, sizeof(int) * cells, st));
        k_cell_of<<<ed_div_up(N, 256), 256, 0, st>>>(P4, N, ctx->misc, ctx->fmisc, ctx->cell_of); ed_note_launch();
        ED_LAUNCH_CHECK();
        for (int ph = 0; ph < 27; ++ph) {
            k_poisson_pick<<<ed_div_up(N, 256), 256, 0, st>>>(P4, N, ph, ctx->misc, ctx->fmisc, ctx->cell_of,
                                                               ctx->cell_node, ctx->cell_pick); ed_note_launch();
            k_poisson_commit<<<1, 1024, 0, st>>>(P4, ph, ctx->misc, ctx->cell_pick, ctx->cell_node, G4, max_nodes); ed_note_launch();
        }
        ED_LAUNCH_CHECK();
        if ((s = read_misc(ctx, hm, st)) != ED_OK) return s;
        const int mt = hm[MI_PHASE_BASE];
        m = mt < max_nodes ? mt : max_nodes;
        int cnt[2] = {m, mt};
        ED_CUDA_TRY(cudaMemcpyAsync(graph->counts, cnt, sizeof(cnt), cudaMemcpyHostToDevice, st));
    } else {
        m = m_in;
        int cnt[2] = {m, m};
        ED_CUDA_TRY(cudaMemcpyAsync(graph->counts, cnt, sizeof(cnt), cudaMemcpyHostToDevice, st));
    }
    if (m < ED_K || (prm->weight_mode == ED_WEIGHT_EQ2 && m < ED_K + 1) || m <= prm->k_graph) return ED_ERR_ARG;

    // ---- nearest nodes and weights ----
    {
        const int kcells = hm[MI_KDIMS + 3];
        ED_CUDA_TRY(cudaMemsetAsync(ctx->kcell_cnt, 0, sizeof(int) * (kcells + 1), st));
        int *cell_of_node = ctx->row_cnt;   // scratch (m + 1 ints)
        k_kcell_count<<<ed_div_up(m, 256), 256, 0, st>>>(G4, m, ctx->misc, ctx->fmisc, ctx->kcell_cnt, cell_of_node); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->kcell_cnt, ctx->kcell_start, kcells, st)) != ED_OK) return s;
        ED_CUDA_TRY(cudaMemsetAsync(ctx->kcell_cnt, 0, sizeof(int) * (kcells + 1), st));
        k_kcell_fill<<<ed_div_up(m, 256), 256, 0, st>>>(m, ctx->kcell_start, ctx->kcell_cnt, cell_of_node,
                                                         ctx->kcell_nodes); ed_note_launch();
        k_knn<<<ed_div_up(N, 128), 128, 0, st>>>(P4, N, G4, m, ctx->misc, ctx->fmisc, ctx->kcell_start,
                                                  ctx->kcell_nodes, prm->weight_mode, prm->sigma,
                                                  (ushort4 *)graph->idx, (float4 *)graph->weights); ed_note_launch();
        k_node_graph<<<ed_div_up(m, 128), 128, 0, st>>>(G4, m, prm->k_graph, graph->nbr); ed_note_launch();
        ED_LAUNCH_CHECK();
    }

    // ---- block pattern ----
    const int words = ed_div_up(m, 32);
    int nnzb;
    {
        ED_CUDA_TRY(cudaMemsetAsync(ctx->bitmap, 0, sizeof(uint32_t) * (size_t)m * words, st));
        k_pairs_points<<<ed_div_up(N, 256), 256, 0, st>>>((const ushort4 *)graph->idx, N, ctx->bitmap, words); ed_note_launch();
        k_pairs_graph<<<ed_div_up(m, 256), 256, 0, st>>>(graph->nbr, m, prm->k_graph, ctx->bitmap, words); ed_note_launch();
        k_row_count<<<ed_div_up(m, 128), 128, 0, st>>>(ctx->bitmap, m, words, ctx->row_cnt); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->row_cnt, ctx->row_ptr, m, st)) != ED_OK) return s;
        ED_CUDA_TRY(cudaMemcpyAsync(&nnzb, ctx->row_ptr + m, sizeof(int), cudaMemcpyDeviceToHost, st));
        ED_CUDA_TRY(cudaStreamSynchronize(st));
        if (nnzb > ctx->max_nnzb) return ED_ERR_CAPACITY;
        k_row_fill<<<ed_div_up(m, 128), 128, 0, st>>>(ctx->bitmap, m, words, ctx->row_ptr, ctx->col, ctx->brow,
                                                      ctx->diag_pos); ed_note_launch();
        k_tpos<<<ed_div_up(nnzb, 256), 256, 0, st>>>(nnzb, ctx->row_ptr, ctx->col, ctx->brow, ctx->tpos, ctx->flag_a); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->flag_a, ctx->flag_b, nnzb, st)) != ED_OK) return s;
        k_compact_upper<<<ed_div_up(nnzb, 256), 256, 0, st>>>(nnzb, ctx->flag_a, ctx->flag_b, ctx->up_list); ed_note_launch();
        ED_LAUNCH_CHECK();
    }

    // ---- per-block point lists (stable: point order inside each block) ----
    const int ne = 10 * N;
    int nchunks, n_upper = 0;
    {
        k_entries_gen<<<ed_div_up(N, 128), 128, 0, st>>>((const ushort4 *)graph->idx, N, ctx->row_ptr, ctx->col,
                                                          ctx->ent_key, ctx->ent_val, ctx->misc + MI_STATUS); ed_note_launch();
        ED_LAUNCH_CHECK();
        int bits = 1;
        while ((1 << bits) < nnzb) ++bits;
        if ((s = ed_radix_sort_pairs(ctx, ctx->ent_key, ctx->ent_val, ne, bits, st)) != ED_OK) return s;
        ED_CUDA_TRY(cudaMemsetAsync(ctx->ent_cnt, 0, sizeof(int) * nnzb, st));
        k_ent_count<<<ed_div_up(ne, 256), 256, 0, st>>>(ctx->ent_key, ne, ctx->ent_cnt); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->ent_cnt, ctx->ent_start, nnzb, st)) != ED_OK) return s;
        k_chunk_count<<<ed_div_up(nnzb, 256), 256, 0, st>>>(nnzb, ctx->ent_cnt, ctx->brow, ctx->col, ctx->chunk_cnt); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->chunk_cnt, ctx->chunk_start, nnzb, st)) != ED_OK) return s;
        ED_CUDA_TRY(cudaMemcpyAsync(&nchunks, ctx->chunk_start + nnzb, sizeof(int), cudaMemcpyDeviceToHost, st));
        if ((s = read_misc(ctx, hm, st)) != ED_OK) return s;
        if (hm[MI_STATUS] != ED_OK) return (ed_status)hm[MI_STATUS];
        if (nchunks > ctx->max_chunks) return ED_ERR_CAPACITY;
        k_chunk_fill<<<ed_div_up(nnzb, 256), 256, 0, st>>>(nnzb, ctx->ent_cnt, ctx->ent_start, ctx->brow, ctx->col,
                                                           ctx->chunk_start, ctx->chunks); ed_note_launch();
        ED_LAUNCH_CHECK();
        int cnt3[2] = {nnzb, 0};
        ED_CUDA_TRY(cudaMemcpyAsync(graph->counts + 2, cnt3, sizeof(cnt3), cudaMemcpyHostToDevice, st));
        ED_CUDA_TRY(cudaMemcpyAsync(&n_upper, ctx->flag_b + nnzb, sizeof(int), cudaMemcpyDeviceToHost, st));
        ED_CUDA_TRY(cudaStreamSynchronize(st));
        if (2 * n_upper != nnzb + m) return ED_ERR_STATE;   // the pattern must be symmetric with a full diagonal
    }

    ctx->pos = pos;
    ctx->nrm = nrm;
    ctx->N = N;
    ctx->graph = *graph;
    ctx->k_graph = prm->k_graph;
    ctx->weight_mode = prm->weight_mode;
    ctx->sigma = prm->sigma;
    ctx->m = m;
    ctx->nnzb = nnzb;
    ctx->n_upper = n_upper;
    ctx->n_entries = ne;
    ctx->n_chunks = nchunks;
    ctx->have_graph = 1;
    return ED_OK;
}
