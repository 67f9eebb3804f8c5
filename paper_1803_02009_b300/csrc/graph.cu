// graph.cu -- ed_build_graph: ED nodes, nearest nodes and weights, node
// graph, and the block structure of the normal equations (Sec. II.D-II.E).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "ed_internal.cuh"

__global__ void k_bbox_init(int *misc)
{
    if (threadIdx.x < 3) {
        misc[MI_BBOX + threadIdx.x] = 0x7fffffff;
        misc[MI_BBOX + 3 + threadIdx.x] = (int)0x80000000;
    }
}

// the first kernel of a build: the misc words cleared (the bounding box at
// its empty extremes) and the count arrays of the tuple buckets and the
// incidences zeroed (grid-stride)
__global__ void k_build_init(int *__restrict__ misc, int *__restrict__ z0, int n0, int *__restrict__ z1, int n1)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int i = t; i < MI_COUNT; i += stride)
        misc[i] = i >= MI_BBOX && i < MI_BBOX + 3 ? 0x7fffffff : (i >= MI_BBOX + 3 && i < MI_BBOX + 6 ? (int)0x80000000 : 0);
    for (int i = t; i < n0; i += stride) z0[i] = 0;
    for (int i = t; i < n1; i += stride) z1[i] = 0;
}

__global__ void __launch_bounds__(256) k_bbox(const float4 *__restrict__ pos, int n, int *misc)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ float smn[3][8], smx[3][8];
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
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            smn[d][w] = mn[d];
            smx[d][w] = mx[d];
        }
    __syncthreads();
    // one atomic per CTA and bound (min/max are exact in any order)
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        float a = smn[d][0], b = smx[d][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            a = fminf(a, smn[d][k]);
            b = fmaxf(b, smx[d][k]);
        }
        atomicMin(&misc[MI_BBOX + d], f2o(a));
        atomicMax(&misc[MI_BBOX + 3 + d], f2o(b));
    }
}

// cell size, inverse and dims of the sampling grid (edge r / sqrt 3) and of the
// search grid (edge kc), by the same FP32 operations as the oracle
__global__ void k_grid_setup(int *misc, float *fmisc, float r, float kc, long max_cells, int sampling)
{
    ed_pdl_wait();
    ed_pdl_trigger();
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

#define NO_BID 0x7f7f7f7f

// every cell of the sampling grid without a bid (the cell count from the set-up)
__global__ void k_fill_cells(int *__restrict__ cell_pick, const int *__restrict__ misc)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (misc[MI_STATUS] != ED_OK) return;
    const int cells = misc[MI_DIMS + 3];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) cell_pick[c] = NO_BID;
}

__global__ void k_cell_of(const float4 *__restrict__ pos, int n, const int *__restrict__ misc,
                          const float *__restrict__ fmisc, int *__restrict__ cell_of)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || misc[MI_STATUS] != ED_OK) return;   // no grid when the set-up failed
    const int dims[3] = {misc[MI_DIMS], misc[MI_DIMS + 1], misc[MI_DIMS + 2]};
    const float4 p = pos[i];
    int3 c = cell3(p.x, p.y, p.z, fmisc, fmisc[MF_INV], dims);
    cell_of[i] = c.x + dims[0] * (c.y + dims[1] * c.z);
}

// Poisson-disk sampling (27 phases).  Points are bucketed by the phase of
// their cell once; phase ph then runs over its bucket only.  A cell's winning
// bid (lowest point index) is the node of that cell: later phases read it
// straight from cell_pick (a cell of a later phase still holds the "no bid"
// pattern 0x7f7f7f7f, and cells of the same phase are never within +-2 cells
// of each other), so no per-phase commit is needed.  Node numbers follow the
// (phase, linear cell index) order and are assigned by one scan at the end.


__device__ __forceinline__ int cell_phase(int c, int nx, int ny)
{
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    return (cx % 3) + 3 * (cy % 3) + 9 * (cz % 3);
}

__global__ void k_phase_count(const int *__restrict__ cell_of, int n, const int *__restrict__ misc,
                              int *__restrict__ cnt)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (misc[MI_STATUS] != ED_OK) return;
    __shared__ int h[27];
    if (threadIdx.x < 27) h[threadIdx.x] = 0;
    __syncthreads();
    const int nx = misc[MI_DIMS], ny = misc[MI_DIMS + 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&h[cell_phase(cell_of[i], nx, ny)], 1);
    __syncthreads();
    if (threadIdx.x < 27 && h[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], h[threadIdx.x]);
}

// exclusive scan of the 27 phase counts (start[27] = n); fill counters cleared
__global__ void k_phase_scan(const int *__restrict__ cnt, int *__restrict__ start, int *__restrict__ fill)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (threadIdx.x != 0) return;
    int s = 0;
    for (int p = 0; p < 27; ++p) {
        start[p] = s;
        s += cnt[p];
        fill[p] = 0;
    }
    start[27] = s;
}

__global__ void k_phase_scatter(const int *__restrict__ cell_of, int n, const int *__restrict__ misc,
                                const int *__restrict__ start, int *__restrict__ fill, int2 *__restrict__ bucket)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (misc[MI_STATUS] != ED_OK) return;
    __shared__ int h[27], base[27];
    const int nx = misc[MI_DIMS], ny = misc[MI_DIMS + 1];
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
        if (threadIdx.x < 27) h[threadIdx.x] = 0;
        __syncthreads();
        const int i = i0 + threadIdx.x;
        int ph = -1, loc = 0, ci = 0;
        if (i < n) {
            ci = cell_of[i];
            ph = cell_phase(ci, nx, ny);
            loc = atomicAdd(&h[ph], 1);
        }
        __syncthreads();
        if (threadIdx.x < 27) base[threadIdx.x] = h[threadIdx.x] ? atomicAdd(&fill[threadIdx.x], h[threadIdx.x]) : 0;
        __syncthreads();
        if (i < n) bucket[start[ph] + base[ph] + loc] = make_int2(i, ci);
        __syncthreads();
    }
}

// phase ph: a point bids for its cell when its FP32 key to every node chosen
// in earlier phases (cells within +-2) is >= r*r; the lowest index wins.
// Five lanes per point (lanes 5g .. 5g+4 of a warp, six points per warp) each
// check one z layer of the 5x5x5 neighbourhood; the group votes.  All 27
// phases run in one persistent cooperative launch with a grid barrier between
// phases; the winning bids of earlier phases are read from L2 (they were
// written by atomics of other CTAs during this launch).
__device__ __forceinline__ void poisson_phase(const float4 *__restrict__ pos, const int2 *__restrict__ bucket, int e0,
                                              int e1, int ph, int nx, int ny, int nz, float r2, int *cell_pick,
                                              int2 first_bc, float4 first_p)
{
    const int lane = threadIdx.x & 31, grp = lane / 5, sub = lane % 5;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    // phase residues of the neighbours at offsets -2..2 (this phase's cells
    // have residues px, py, pz): only cells of earlier phases can hold a node
    const int px = ph % 3, py = (ph / 3) % 3, pz = ph / 9;
    int rx[5], ry[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        rx[d] = (px + d + 1) % 3;
        ry[d] = 3 * ((py + d + 1) % 3);
    }
    bool first = true;
    for (int wbase = e0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 6; wbase < e1; wbase += warps * 6) {
        const int e = wbase + grp;
        const bool act = grp < 6 && e < e1;
        bool ok = true;
        int i = -1, c = 0;
        if (act) {
            // the first round's bucket entry and point were loaded before the barrier
            const int2 bc = first ? first_bc : bucket[e];
            i = bc.x;
            c = bc.y;
            const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
            const int dz = sub - 2, az = cz + dz;
            const int rz = 9 * ((pz + sub + 1) % 3);
            if (az >= 0 && az < nz) {
                const float4 p = first ? first_p : pos[i];
                int q[25];
#pragma unroll
                for (int k = 0; k < 25; ++k) {
                    const int ay = cy + k / 5 - 2, ax = cx + k % 5 - 2;
                    // (a cell of this phase or a later one holds no node yet: not read)
                    const bool in = ay >= 0 && ay < ny && ax >= 0 && ax < nx && !(dz == 0 && k == 12) &&
                                    rx[k % 5] + ry[k / 5] + rz < ph;
                    q[k] = in ? __ldcg(cell_pick + ax + nx * (ay + ny * az)) : NO_BID;   // earlier phases: final
                }
#pragma unroll
                for (int k = 0; k < 25; ++k) {
                    if (q[k] == NO_BID) continue;
                    const float4 g = pos[q[k]];
                    if (ed_key(p.x, p.y, p.z, g.x, g.y, g.z) < r2) ok = false;
                }
            }
        }
        first = false;
        // the group's vote: every one of its five lanes found no close node
        const unsigned bad = __ballot_sync(0xffffffffu, act && !ok);
        const unsigned gmask = 0x1fu << (5 * grp);
        if (act && sub == 0 && !(bad & gmask)) atomicMin(&cell_pick[c], i);
    }
}

// the bucket entry and point of this lane's group in the first round of a
// phase (independent of the picks, so loaded before the barrier that opens it)
__device__ __forceinline__ void poisson_prefetch(const float4 *__restrict__ pos, const int2 *__restrict__ bucket,
                                                 int e0, int e1, int2 &bc, float4 &p)
{
    const int lane = threadIdx.x & 31, grp = lane / 5;
    const int e = e0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 6 + grp;
    bc = make_int2(0, 0);
    p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (grp < 6 && e < e1) {
        bc = bucket[e];
        p = pos[bc.x];
    }
}

#define POISSON_T 512
__global__ void __launch_bounds__(POISSON_T) k_poisson_all(const float4 *__restrict__ pos, const int2 *__restrict__ bucket,
                                                           const int *__restrict__ start, const int *__restrict__ misc_in,
                                                           const float *__restrict__ fmisc, int *cell_pick, unsigned *bar,
                                                           int *status, unsigned long long wait_ns)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ int s_flag;
    if (*(volatile int *)status != ED_OK) return;   // every CTA: no grid when the set-up failed
    const int nx = misc_in[MI_DIMS], ny = misc_in[MI_DIMS + 1], nz = misc_in[MI_DIMS + 2];
    const float r2 = fmisc[MF_R2];
    unsigned target = 0;
    int2 bc;
    float4 p;
    poisson_prefetch(pos, bucket, start[0], start[1], bc, p);
    for (int ph = 0; ph < 27; ++ph) {
        poisson_phase(pos, bucket, start[ph], start[ph + 1], ph, nx, ny, nz, r2, cell_pick, bc, p);
        if (ph < 26) {
            poisson_prefetch(pos, bucket, start[ph + 1], start[ph + 2], bc, p);
            if (!ed_grid_sync(bar, status, gridDim.x, target, &s_flag, wait_ns)) return;
        }
    }
}

struct PhaseTable {
    int off[28];   // first enumeration index of every phase (cells in phase-major order)
    int ax[27], ay[27];
};

__device__ __forceinline__ int phase_cell(const PhaseTable &T, int t, int nx, int ny, int &ph)
{
    int p = 0;
    while (p < 26 && t >= T.off[p + 1]) ++p;
    ph = p;
    const int k = t - T.off[p];
    const int a = k % T.ax[p], b = (k / T.ax[p]) % T.ay[p], c = k / (T.ax[p] * T.ay[p]);
    return (p % 3 + 3 * a) + nx * (((p / 3) % 3 + 3 * b) + ny * (p / 9 + 3 * c));
}

__global__ void k_node_flags(PhaseTable T, int total, const int *__restrict__ misc, const int *__restrict__ cell_pick,
                             int *__restrict__ flag)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int ph;
    const int L = phase_cell(T, t, misc[MI_DIMS], misc[MI_DIMS + 1], ph);
    flag[t] = cell_pick[L] != NO_BID;
}

__global__ void k_node_write(PhaseTable T, int total, const int *__restrict__ misc, const int *__restrict__ cell_pick,
                             const int *__restrict__ pre, const float4 *__restrict__ pos, float4 *__restrict__ nodes,
                             int max_nodes)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total || pre[t + 1] == pre[t]) return;
    const int id = pre[t];
    if (id >= max_nodes) return;
    int ph;
    const int L = phase_cell(T, t, misc[MI_DIMS], misc[MI_DIMS + 1], ph);
    const float4 p = pos[cell_pick[L]];
    nodes[id] = make_float4(p.x, p.y, p.z, 0.f);
}

// ---------------------------------------------------------------------------
// nearest-node search grid
// ---------------------------------------------------------------------------

// (m, the node count, is read from the graph's counts: the launches are queued
// before the host knows it)
__global__ void k_kcell_count(const float4 *__restrict__ nodes, const int *__restrict__ m_dev,
                              const int *__restrict__ misc, const float *__restrict__ fmisc, int *__restrict__ cnt,
                              int *__restrict__ cell_of_node)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *m_dev) return;
    const int dims[3] = {misc[MI_KDIMS], misc[MI_KDIMS + 1], misc[MI_KDIMS + 2]};
    const float4 g = nodes[j];
    int3 c = cell3(g.x, g.y, g.z, fmisc, fmisc[MF_KINV], dims);
    const int L = c.x + dims[0] * (c.y + dims[1] * c.z);
    cell_of_node[j] = L;
    atomicAdd(&cnt[L], 1);
}

// every node's position, its index in w (as int bits), in its search cell's
// range, the slots taken by counting the cell's count down to 0 (the order
// inside a cell is immaterial: the search orders by key and index)
__global__ void k_kcell_fill(const int *__restrict__ m_dev, const float4 *__restrict__ nodes,
                             const int *__restrict__ start, int *__restrict__ fill, const int *__restrict__ cell_of_node,
                             float4 *__restrict__ kpos)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *m_dev) return;
    const int L = cell_of_node[j];
    const float4 g = nodes[j];
    kpos[start[L] + atomicSub(&fill[L], 1) - 1] = make_float4(g.x, g.y, g.z, __int_as_float(j));
}

#define KNN_S 5   // K + 1 nearest (Eq. 2 needs the (K+1)-th distance)

// insertion of (key, id) into the sorted list (kk, ii) of the KNN_S best
// (ties to the lower index): the new entry replaces the last one and moves up
// by compare-exchanges with static indices, so the lists stay in registers
__device__ __forceinline__ void topk_ins(float (&kk)[KNN_S], int (&ii)[KNN_S], float key, int id)
{
    if (key > kk[KNN_S - 1] || (key == kk[KNN_S - 1] && id >= ii[KNN_S - 1])) return;
    kk[KNN_S - 1] = key;
    ii[KNN_S - 1] = id;
#pragma unroll
    for (int p = KNN_S - 1; p > 0; --p) {
        const bool up = kk[p - 1] > kk[p] || (kk[p - 1] == kk[p] && ii[p - 1] > ii[p]);
        const float tk = kk[p - 1];
        const int ti = ii[p - 1];
        kk[p - 1] = up ? kk[p] : tk;
        ii[p - 1] = up ? ii[p] : ti;
        kk[p] = up ? tk : kk[p];
        ii[p] = up ? ti : ii[p];
    }
}

// kk[q] for a run-time q < KNN_S, by static indices
__device__ __forceinline__ float pick_k(const float (&kk)[KNN_S], int q)
{
    float v = kk[0];
#pragma unroll
    for (int s = 1; s < KNN_S; ++s) v = q == s ? kk[s] : v;
    return v;
}

// K+1 nearest nodes by rings of search cells; a ring R is the last one needed
// once the (K+1)-th key is below (R * cell)^2 (with a round-off margin): every
// node outside rings 0..R is at least R cells away.  Then the weights.
__global__ void k_knn(const float4 *__restrict__ pos, int n, const float4 *__restrict__ nodes,
                      const int *__restrict__ m_dev, const int *__restrict__ misc, const float *__restrict__ fmisc,
                      const int *__restrict__ start, const float4 *__restrict__ kpos, int mode, float sigma,
                      ushort4 *__restrict__ idx_out, float4 *__restrict__ w_out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int m = *m_dev;
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
    // rings 0 and 1 together (the stopping test after ring 0 never holds: its
    // bound is 0), as the nine x-rows of the 3x3x3 block: each row is one
    // contiguous range of the cell-sorted nodes, and every range bound is loaded
    // before the first node (the order of the candidates does not change the
    // result: the lists are ordered by key and index)
    {
        int lo[9], hi[9];
        const int x0 = c.x > 0 ? c.x - 1 : 0, x1 = c.x + 1 < dims[0] ? c.x + 1 : dims[0] - 1;
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const int ay = c.y + (r % 3) - 1, az = c.z + (r / 3) - 1;
            const bool ok = ay >= 0 && ay < dims[1] && az >= 0 && az < dims[2];
            const int Lb = dims[0] * (ay + dims[1] * az);
            lo[r] = ok ? start[Lb + x0] : 0;
            hi[r] = ok ? start[Lb + x1 + 1] : 0;
        }
#pragma unroll
        for (int r = 0; r < 9; ++r)
            for (int t = lo[r]; t < hi[r]; ++t) {
                const float4 g = __ldg(kpos + t);
                topk_ins(kk, ii, ed_key(p.x, p.y, p.z, g.x, g.y, g.z), __float_as_int(g.w));
            }
    }
    bool done = false;
    if (need > 0) {
        const float kn = pick_k(kk, need - 1);
        done = kn < INFINITY && kn < kc * kc * 0.99999f;
    }
    for (int R = 2; R <= maxR && !done; ++R) {
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
                            const float4 g = __ldg(kpos + t);
                            topk_ins(kk, ii, ed_key(p.x, p.y, p.z, g.x, g.y, g.z), __float_as_int(g.w));
                        }
                    }
                    if (R == 0) break;
                }
            }
        }
        if (need > 0) {
            const float kn = pick_k(kk, need - 1);
            const float b = (float)R * kc;
            if (kn < INFINITY && kn < b * b * 0.99999f) break;
        }
    }
    // weights (Eq. 1 normalised; Gaussian or Eq. 2); slots >= m hold no node
    float4 wv;
    if (mode == ED_WEIGHT_GAUSSIAN) {
        wv = ed_gauss_weights_from_keys(kk, m < 4 ? m : 4, sigma);
    } else {
        float w[4], sum = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float t;
            if (ii[s] == 0x7fffffff) t = 0.f;
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
        wv = make_float4(w[0], w[1], w[2], w[3]);
    }
    unsigned short id4[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) id4[s] = (unsigned short)(ii[s] == 0x7fffffff ? 0 : ii[s]);
    idx_out[i] = make_ushort4(id4[0], id4[1], id4[2], id4[3]);
    w_out[i] = wv;
}

// N(j): the k_graph nearest other nodes (FP32 key, ties to the lower index).
// One warp per node: every lane keeps the best k_graph of its strided share of
// the nodes, then the warp merges the 32 sorted lists by repeated minimum of
// (key bits, index) -- keys are non-negative, so their bits order like floats.
// The candidates come from shared memory, NG_TILE nodes at a time.
#define NG_WARPS 16
#define NG_TILE 2048
__global__ void __launch_bounds__(32 * NG_WARPS) k_node_graph(const float4 *__restrict__ nodes,
                                                              const int *__restrict__ m_dev, int kg,
                                                              int *__restrict__ nbr, uint32_t *__restrict__ bm,
                                                              int bm_n)
{
    __shared__ float4 s_nodes[NG_TILE];
    // the pair bitmap of the block pattern zeroed for this build (its first
    // bm_n words: every row of the node count's stride)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bm_n; i += gridDim.x * blockDim.x) bm[i] = 0u;
    const int m = *m_dev;
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * NG_WARPS + (threadIdx.x >> 5);
    const bool active = j < m;
    unsigned long long best[ED_MAX_KG];
    for (int s = 0; s < ED_MAX_KG; ++s) best[s] = ~0ull;
    const float4 g = active ? nodes[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t0 = 0; t0 < m; t0 += NG_TILE) {
        const int tn = min(NG_TILE, m - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < tn; i += 32 * NG_WARPS) s_nodes[i] = __ldg(nodes + t0 + i);
        __syncthreads();
        if (!active) continue;
        for (int li = lane; li < tn; li += 32) {
            const int l = t0 + li;
            if (l == j) continue;
            const float4 h = s_nodes[li];
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(ed_key(g.x, g.y, g.z, h.x, h.y, h.z)) << 32) | (unsigned)l;
            if (key >= best[kg - 1]) continue;
            int p = kg - 1;
            while (p > 0 && best[p - 1] > key) {
                best[p] = best[p - 1];
                --p;
            }
            best[p] = key;
        }
    }
    if (!active) return;
    int head = 0;
    for (int s = 0; s < kg; ++s) {
        const unsigned long long mine = head < kg ? best[head] : ~0ull;
        unsigned long long mn = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, mn, o);
            mn = other < mn ? other : mn;
        }
        if (mine == mn && mn != ~0ull) ++head;   // (key, index) pairs are unique: one lane pops
        if (lane == 0) nbr[j * kg + s] = mn == ~0ull ? -1 : (int)(mn & 0xffffffffu);
    }
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

// the same with the run count read from the device (queued before the host has it)
__global__ void k_pairs_runs_dev(const int *__restrict__ n_runs_dev, const int *__restrict__ run_start,
                                 const ushort4 *__restrict__ sidx, uint32_t *bm, int words)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *n_runs_dev) return;
    const ushort4 q = sidx[run_start[r]];
    const int id[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (a != b) set_bit(bm, words, id[a], id[b]);
}

__global__ void k_pairs_graph(const int *__restrict__ nbr, int m, int kg, uint32_t *bm, int words)
{
    ed_pdl_wait();
    ed_pdl_trigger();
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

// one warp per node row: the set bits of its bitmap words
__global__ void k_row_count(const uint32_t *__restrict__ bm, int m, int words, int *__restrict__ cnt)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= m) return;
    int c = 0;
    for (int w = lane; w < words; w += 32) c += __popc(bm[(long)j * words + w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[j] = c;
}

// (queued before the host has the block count: a count above the capacity
// writes nothing and sets the status)
__global__ void k_row_fill(const uint32_t *__restrict__ bm, int m, int words, const int *__restrict__ row_ptr,
                           int *__restrict__ col, int *__restrict__ brow, int *__restrict__ diag_pos, int max_nnzb,
                           int *__restrict__ status)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    // one warp per node row: the words in rounds of 32, a lane's bits placed
    // after the bits of the lanes (and rounds) before it: ascending columns
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row_ptr[m] > max_nnzb) {
        if (j == 0 && lane == 0) atomicCAS(status, ED_OK, ED_ERR_CAPACITY);
        return;
    }
    if (j >= m) return;
    int p = row_ptr[j];
    for (int w0 = 0; w0 < words; w0 += 32) {
        const int w = w0 + lane;
        uint32_t v = w < words ? bm[(long)j * words + w] : 0u;
        const int c = __popc(v);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int q = p + incl - c;
        while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1;
            const int l = (w << 5) + b;
            if (l == j) diag_pos[j] = q;
            col[q] = l;
            brow[q] = j;
            ++q;
        }
        p += __shfl_sync(0xffffffffu, incl, 31);
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

// (the block count nnzb is read on the device; nothing runs when it exceeds
// the capacity -- the row fill has reported ED_ERR_CAPACITY then)
__global__ void k_tpos(const int *__restrict__ nnzb_dev, int cap, const int *__restrict__ row_ptr,
                       const int *__restrict__ col, const int *__restrict__ brow, int *__restrict__ tpos,
                       int *__restrict__ upper_flag)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int nnzb = *nnzb_dev;
    if (nnzb > cap) return;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nnzb; b += gridDim.x * blockDim.x) {
        const int j = brow[b], l = col[b];
        tpos[b] = find_block(row_ptr, col, l, j);
        upper_flag[b] = l > j;   // strictly upper: the diagonal blocks go first in the list
    }
}

// finalisation work list: the m diagonal blocks (long warps) first, then the
// strictly upper blocks in row order
__global__ void k_compact_upper(const int *__restrict__ nnzb_dev, int cap, int m, const int *__restrict__ flag,
                                const int *__restrict__ pre, const int *__restrict__ diag_pos,
                                int *__restrict__ up_list)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int nnzb = *nnzb_dev;
    if (nnzb > cap) return;
    const int n = nnzb > m ? nnzb : m;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        if (b < m) up_list[b] = diag_pos[b];
        if (b < nnzb && flag[b]) up_list[m + pre[b]] = b;
    }
}

// ---------------------------------------------------------------------------
// points grouped by their node tuple.  Every point carries its k = 4 nearest
// nodes; the points whose four nodes are the same set form a run of the
// points sorted by that set (the tuple, nodes in increasing index order).  A
// run contributes to the 10 blocks (tuple[s], tuple[t]), s <= t, of J^T J;
// each such (block, run) pair is an incidence, and the assembly streams, for
// one block, the points of its runs.
// ---------------------------------------------------------------------------

// the four nodes of a point in increasing index order, with the slot (position
// in the point's nearest-node list) each came from: a sorting network
__device__ __forceinline__ void tuple_of(ushort4 q, int (&n)[4], int (&slot)[4])
{
    n[0] = q.x; n[1] = q.y; n[2] = q.z; n[3] = q.w;
    slot[0] = 0; slot[1] = 1; slot[2] = 2; slot[3] = 3;
    auto cx = [&](int a, int b) {
        if (n[a] > n[b]) {
            const int t = n[a]; n[a] = n[b]; n[b] = t;
            const int u = slot[a]; slot[a] = slot[b]; slot[b] = u;
        }
    };
    cx(0, 1); cx(2, 3); cx(0, 2); cx(1, 3); cx(1, 2);
}

// sort key of a tuple: the four indices in fields of `fb` bits, the smallest
// node most significant
__device__ __forceinline__ unsigned long long tuple_key(const int (&n)[4], int fb)
{
    return ((unsigned long long)n[0] << (3 * fb)) | ((unsigned long long)n[1] << (2 * fb)) |
           ((unsigned long long)n[2] << fb) | (unsigned long long)n[3];
}

// ---- grouping by bucket sort: the points are counted into buckets by their
// tuple's smallest node, placed (in any order) into their bucket's range,
// and each bucket is then ordered by the rest of the tuple and the point
// index.  The order equals that of a stable sort by the full tuple key. ----

// the lanes of a warp with the same bucket add their count with one atomic:
// returns each lane's position among the warp's lanes of its bucket, and the
// bucket's base from the atomic (fill pass) or nothing (count pass)
__device__ __forceinline__ int warp_bucket_add(int *ctr, int bucket, bool active)
{
    const unsigned peers = __match_any_sync(0xffffffffu, active ? bucket : -1);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (active && lane == leader) base = atomicAdd(ctr + bucket, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void k_tb_count(const ushort4 *__restrict__ idx, int n, int *__restrict__ cnt)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int t[4] = {0, 0, 0, 0}, sl[4];
    if (i < n) tuple_of(idx[i], t, sl);
    warp_bucket_add(cnt, t[0], i < n);
}

__global__ void k_tb_place(const ushort4 *__restrict__ idx, int n, const int *__restrict__ start,
                           int *__restrict__ fill, uint32_t *__restrict__ order)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int t[4] = {0, 0, 0, 0}, sl[4];
    if (i < n) tuple_of(idx[i], t, sl);
    const int pos = warp_bucket_add(fill, t[0], i < n);
    if (i < n) order[start[t[0]] + pos] = (uint32_t)i;
}

// one CTA per bucket: its points ordered by (the other three nodes, point
// index) -- unique keys -- by a bitonic sort in shared memory over the
// bucket padded to a power of two (TB_MAX at most); a larger bucket by ranks
// against shared-memory tiles instead
#define TB_T 256
#define TB_MAX 2048
// The same ordering with the key and the point index packed into one 64-bit
// word (rest of the tuple << pb | point: unique, so the order is total; for
// 3 fb + pb <= 64): one compare-exchange pair per thread and step of the
// bitonic network (TB64_T = 512 threads: the largest buckets, near 700
// entries padded to 1024, take every thread once per step; with 128 threads
// those CTAs ran four passes per step and set the kernel's length), and one
// 8-byte array in shared memory.
// Buckets above TB_MAX entries are ranked: every entry counts the smaller
// keys, in tiles of TB_MAX.
#define TB64_T 512
__global__ void __launch_bounds__(TB64_T) k_tb_sort64(const ushort4 *__restrict__ idx, const int *__restrict__ start,
                                                      int nb, int fb, int pb, const uint32_t *__restrict__ order,
                                                      uint32_t *__restrict__ out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ unsigned long long s_k[TB_MAX];
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int b0 = start[b], n = start[b + 1] - b0;
    if (n == 0) return;
    if (n == 1) {
        if (threadIdx.x == 0) out[b0] = order[b0];
        return;
    }
    const unsigned long long pmask = (1ull << pb) - 1ull;
    auto packed = [&](uint32_t i) {
        int t[4], sl[4];
        tuple_of(idx[i], t, sl);
        const unsigned long long k3 =
            ((unsigned long long)t[1] << (2 * fb)) | ((unsigned long long)t[2] << fb) | (unsigned long long)t[3];
        return (k3 << pb) | (unsigned long long)i;
    };
    if (n <= TB_MAX) {
        int P = 2;
        while (P < n) P <<= 1;
        for (int q = threadIdx.x; q < P; q += TB64_T) s_k[q] = q < n ? packed(order[b0 + q]) : ~0ull;   // padding last
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < (P >> 1); i += TB64_T) {
                    const int q = ((i & ~(j - 1)) << 1) | (i & (j - 1)), o = q | j;
                    const bool up = (q & k) == 0;
                    const unsigned long long kq = s_k[q], ko = s_k[o];
                    if ((kq > ko) == up) {
                        s_k[q] = ko;
                        s_k[o] = kq;
                    }
                }
                __syncthreads();
            }
        for (int q = threadIdx.x; q < n; q += TB64_T) out[b0 + q] = (uint32_t)(s_k[q] & pmask);
        return;
    }
    for (int e0 = 0; e0 < n; e0 += TB64_T) {
        const int e = e0 + threadIdx.x;
        const unsigned long long ke = e < n ? packed(order[b0 + e]) : 0ull;
        int rank = 0;
        for (int t0 = 0; t0 < n; t0 += TB_MAX) {
            __syncthreads();
            for (int q = threadIdx.x; q < TB_MAX && t0 + q < n; q += TB64_T) s_k[q] = packed(order[b0 + t0 + q]);
            __syncthreads();
            if (e < n) {
                const int lim = min(TB_MAX, n - t0);
                for (int q = 0; q < lim; ++q) rank += s_k[q] < ke;
            }
        }
        if (e < n) out[b0 + rank] = (uint32_t)(ke & pmask);
    }
}

__global__ void __launch_bounds__(TB_T) k_tb_sort(const ushort4 *__restrict__ idx, const int *__restrict__ start,
                                                  int nb, int fb, const uint32_t *__restrict__ order,
                                                  uint32_t *__restrict__ out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ unsigned long long s_key[TB_MAX];
    __shared__ uint32_t s_pt[TB_MAX];
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int b0 = start[b], n = start[b + 1] - b0;
    if (n == 0) return;
    auto key3 = [&](uint32_t i) {
        int t[4], sl[4];
        tuple_of(idx[i], t, sl);
        return ((unsigned long long)t[1] << (2 * fb)) | ((unsigned long long)t[2] << fb) | (unsigned long long)t[3];
    };
    // (key, point) before (key', point')
    auto less = [](unsigned long long ka, uint32_t pa, unsigned long long kb, uint32_t pb) {
        return ka < kb || (ka == kb && pa < pb);
    };
    if (n == 1) {
        if (threadIdx.x == 0) out[b0] = order[b0];
        return;
    }
    if (n <= TB_MAX) {
        int P = 2;
        while (P < n) P <<= 1;
        for (int q = threadIdx.x; q < P; q += TB_T) {
            if (q < n) {
                const uint32_t pq = order[b0 + q];
                s_pt[q] = pq;
                s_key[q] = key3(pq);
            } else {   // padding sorts last
                s_pt[q] = 0xffffffffu;
                s_key[q] = ~0ull;
            }
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = threadIdx.x; q < P; q += TB_T) {
                    const int o = q ^ j;
                    if (o > q) {
                        const bool up = (q & k) == 0;
                        const unsigned long long kq = s_key[q], ko = s_key[o];
                        const uint32_t pq = s_pt[q], po = s_pt[o];
                        if (less(ko, po, kq, pq) == up) {
                            s_key[q] = ko;
                            s_key[o] = kq;
                            s_pt[q] = po;
                            s_pt[o] = pq;
                        }
                    }
                }
                __syncthreads();
            }
        for (int q = threadIdx.x; q < n; q += TB_T) out[b0 + q] = s_pt[q];
        return;
    }
    for (int e0 = 0; e0 < n; e0 += TB_T) {
        const int e = e0 + threadIdx.x;
        uint32_t pi = 0;
        unsigned long long ki = 0;
        if (e < n) {
            pi = order[b0 + e];
            ki = key3(pi);
        }
        int rank = 0;
        for (int t0 = 0; t0 < n; t0 += TB_MAX) {
            __syncthreads();
            for (int q = threadIdx.x; q < TB_MAX && t0 + q < n; q += TB_T) {
                const uint32_t pq = order[b0 + t0 + q];
                s_pt[q] = pq;
                s_key[q] = key3(pq);
            }
            __syncthreads();
            if (e < n) {
                const int lim = min(TB_MAX, n - t0);
                for (int q = 0; q < lim; ++q) rank += less(s_key[q], s_pt[q], ki, pi);
            }
        }
        if (e < n) out[b0 + rank] = pi;
    }
}

// the incidences of every block in run order: counted by block, placed (in
// any order), then each block's short list ordered by run (a run meets a
// block at most once)
// (10 incidences per run, the run count read on the device; a warp's lanes
// take consecutive incidences, so every warp runs the same trip count)
__global__ void k_ic_count(const int *__restrict__ nruns_dev, const int *__restrict__ nnzb_dev, int cap,
                           const uint32_t *__restrict__ key, int *__restrict__ cnt)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (*nnzb_dev > cap) return;
    const int ne = 10 * *nruns_dev;
    for (int e0 = blockIdx.x * blockDim.x; e0 < ne; e0 += gridDim.x * blockDim.x) {
        const int e = e0 + threadIdx.x;
        warp_bucket_add(cnt, e < ne ? (int)key[e] : 0, e < ne);
    }
}

__global__ void k_ic_place(const int *__restrict__ nruns_dev, const int *__restrict__ nnzb_dev, int cap,
                           const uint32_t *__restrict__ key, const uint32_t *__restrict__ val,
                           const int *__restrict__ start, int *__restrict__ fill, uint32_t *__restrict__ out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (*nnzb_dev > cap) return;
    const int ne = 10 * *nruns_dev;
    for (int e0 = blockIdx.x * blockDim.x; e0 < ne; e0 += gridDim.x * blockDim.x) {
        const int e = e0 + threadIdx.x;
        const int b = e < ne ? (int)key[e] : 0;
        const int pos = warp_bucket_add(fill, b, e < ne);
        if (e < ne) out[start[b] + pos] = val[e];
    }
}

// one warp per block: up to 64 incidences (two per lane) by a bitonic sort
// over the warp on the run field; longer lists (rare) by insertion in place
__device__ __forceinline__ void ic_sort_block(const int *__restrict__ start, uint32_t *__restrict__ list, int b,
                                              int lane)
{
    const int b0 = start[b], n = start[b + 1] - b0;
    if (n <= 1) return;
    if (n > 64) {
        if (lane == 0)
            for (int i = 1; i < n; ++i) {
                const uint32_t v = list[b0 + i];
                int j = i - 1;
                while (j >= 0 && (list[b0 + j] >> 4) > (v >> 4)) {
                    list[b0 + j + 1] = list[b0 + j];
                    --j;
                }
                list[b0 + j + 1] = v;
            }
        return;
    }
    // element q of 64 is held by lane q >> 1, slot q & 1; padding sorts last.
    // The network spans the P = 2^k >= n first elements only (the others are
    // padding, and a compare-exchange never pairs q < P with q >= P): a block
    // holds 7.5 runs on average at 640x480
    uint32_t v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) v[u] = 2 * lane + u < n ? list[b0 + 2 * lane + u] : 0xffffffffu;
    int P = 2;
    while (P < n) P <<= 1;
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            // the partners' values, all read before any slot changes: for j = 1
            // the other slot of this lane, else lane ^ (j / 2), same slot
            uint32_t w[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) w[u] = j == 1 ? v[u ^ 1] : __shfl_xor_sync(0xffffffffu, v[u], j >> 1);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int q = 2 * lane + u, o = q ^ j;
                const bool up = (q & k) == 0, lower = q < o;
                // lower element of an ascending pair keeps the smaller run, and so on
                // (padding 0xffffffff has the largest run field)
                const bool take = lower ? ((w[u] >> 4) < (v[u] >> 4)) == up : ((v[u] >> 4) < (w[u] >> 4)) == up;
                if (take) v[u] = w[u];
            }
        }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (2 * lane + u < n) list[b0 + 2 * lane + u] = v[u];
}

// (warps over the blocks, the block count read on the device)
__global__ void __launch_bounds__(128) k_ic_sort(const int *__restrict__ nnzb_dev, int cap,
                                                 const int *__restrict__ start, uint32_t *__restrict__ list,
                                                 const int *__restrict__ brow, const int *__restrict__ col,
                                                 int *__restrict__ bins)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int nnzb = *nnzb_dev;
    if (nnzb > cap) return;
    // and the off-diagonal upper blocks per incidence-count class (the order
    // of the assembly records, k_fin_pack)
    __shared__ int h[ED_ASM_BINS];
    for (int q = threadIdx.x; q < ED_ASM_BINS; q += blockDim.x) h[q] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nnzb; b += (gridDim.x * blockDim.x) >> 5) {
        ic_sort_block(start, list, b, lane);
        if (lane == 0 && brow[b] < col[b]) {
            const int ni = start[b + 1] - start[b];
            atomicAdd(&h[ni < ED_ASM_BINS - 1 ? ni : ED_ASM_BINS - 1], 1);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ED_ASM_BINS; q += blockDim.x)
        if (h[q]) atomicAdd(&bins[q], h[q]);
}

// low 32 bits of every point's key, value = point index (the first pass of a
// two-pass stable sort by the full key)
__global__ void k_tuple_lo(const ushort4 *__restrict__ idx, int n, int fb, uint32_t *__restrict__ key,
                           uint32_t *__restrict__ val)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int t[4], sl[4];
    tuple_of(idx[i], t, sl);
    key[i] = (uint32_t)tuple_key(t, fb);
    val[i] = (uint32_t)i;
}

// high bits of the key of the point at each position of the first pass
__global__ void k_tuple_hi(const ushort4 *__restrict__ idx, int n, int fb, const uint32_t *__restrict__ val,
                           uint32_t *__restrict__ key)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int t[4], sl[4];
    tuple_of(idx[val[e]], t, sl);
    key[e] = (uint32_t)(tuple_key(t, fb) >> 32);
}

// the points in tuple order (sorted position k holds point perm[k]): position,
// normal, the tuple and the skinning weights in tuple order; flag[k] = 1 where
// a run starts
__global__ void k_tuple_gather(const uint32_t *__restrict__ val, int n, const ushort4 *__restrict__ idx,
                               const float4 *__restrict__ w, const float4 *__restrict__ pos,
                               const float4 *__restrict__ nrm, int *__restrict__ perm, float4 *__restrict__ spos,
                               float4 *__restrict__ snrm, ushort4 *__restrict__ sidx, float4 *__restrict__ sw,
                               ushort4 *__restrict__ sidx_d, float4 *__restrict__ sw_d, int *__restrict__ flag)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)val[k];
    const ushort4 id = idx[i];
    int t[4], sl[4];
    tuple_of(id, t, sl);
    const float4 wi = w[i];
    const float wv[4] = {wi.x, wi.y, wi.z, wi.w};
    perm[k] = i;
    spos[k] = pos[i];
    snrm[k] = nrm[i];
    sidx[k] = make_ushort4((unsigned short)t[0], (unsigned short)t[1], (unsigned short)t[2], (unsigned short)t[3]);
    sw[k] = make_float4(wv[sl[0]], wv[sl[1]], wv[sl[2]], wv[sl[3]]);
    sidx_d[k] = id;   // (nearest first, as the graph holds them: the warp's summation order)
    sw_d[k] = wi;
    int start = 1;
    if (k > 0) {
        int tp[4], sp[4];
        tuple_of(idx[val[k - 1]], tp, sp);
        start = tp[0] != t[0] || tp[1] != t[1] || tp[2] != t[2] || tp[3] != t[3];
    }
    flag[k] = start;
}

// run r covers sorted positions [run_start[r], run_start[r + 1]); run_start[n_runs] = n;
// run_of_start[k] = r where k starts run r, -1 elsewhere
__global__ void k_run_starts(const int *__restrict__ flag, const int *__restrict__ pre, int n,
                             int *__restrict__ run_start, int *__restrict__ run_of_start)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    run_of_start[k] = flag[k] ? pre[k] : -1;
    if (flag[k]) run_start[pre[k]] = k;
    if (k == n - 1) run_start[pre[n]] = n;
}

// the 10 incidences of every run: key = block of (tuple[s], tuple[t]) in the
// BSR pattern, value = run << 4 | s << 2 | t (s <= t, so tuple[s] is the row
// node: the block is upper or diagonal)
// the ten incidences of run r: the blocks (t4[s], t4[t]), s <= t, of its
// tuple, found by ten binary searches in the rows of the tuple's nodes that
// advance in step (the loads of one step are independent: about log2(row
// length) rounds of loads instead of ten searches one after another)
__device__ __forceinline__ void inc_gen_run(int r, const int *__restrict__ run_start, const ushort4 *__restrict__ sidx,
                                            const int *__restrict__ row_ptr, const int *__restrict__ col,
                                            uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                                            int *__restrict__ status)
{
    const ushort4 q = sidx[run_start[r]];
    const int t4[4] = {q.x, q.y, q.z, q.w};
    int r0[4], r1[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        r0[s] = row_ptr[t4[s]];
        r1[s] = row_ptr[t4[s] + 1];
    }
    // search e = (s, t): the largest position of row t4[s] whose column is <= t4[t]
    int base[10], len[10], tgt[10];
    {
        int e = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int t = s; t < 4; ++t) {
                base[e] = r0[s];
                len[e] = r1[s] - r0[s];
                tgt[e] = t4[t];
                ++e;
            }
    }
    for (;;) {
        bool more = false;
#pragma unroll
        for (int e = 0; e < 10; ++e) {
            if (len[e] > 1) {
                const int half = len[e] >> 1;
                if (col[base[e] + half] <= tgt[e]) base[e] += half;
                len[e] -= half;
                more = true;
            }
        }
        if (!more) break;
    }
    int e = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = s; t < 4; ++t) {
            const int b = len[e] == 1 && col[base[e]] == tgt[e] ? base[e] : -1;
            if (b < 0) atomicCAS(status, ED_OK, ED_ERR_STATE);
            key[10L * r + e] = (uint32_t)(b < 0 ? 0 : b);
            val[10L * r + e] = ((uint32_t)r << 4) | ((uint32_t)s << 2) | (uint32_t)t;
            ++e;
        }
}

__global__ void k_inc_gen(const int *__restrict__ nruns_dev, const int *__restrict__ nnzb_dev, int cap,
                          const int *__restrict__ run_start, const ushort4 *__restrict__ sidx,
                          const int *__restrict__ row_ptr, const int *__restrict__ col, uint32_t *__restrict__ key,
                          uint32_t *__restrict__ val, int *__restrict__ status)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    if (*nnzb_dev > cap) return;
    const int n_runs = *nruns_dev;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_runs; r += gridDim.x * blockDim.x)
        inc_gen_run(r, run_start, sidx, row_ptr, col, key, val, status);
}



// the assembly's record of every upper block u, fixed for the frame (one load
// for what its warps would otherwise fetch in dependent steps):
//   off-diagonal: {b, j, l, transpose position}, {first incidence, incidences,
//                 graph-edge flags (j -> l: 1, l -> j: 2), 0}
//   diagonal:     {b, j, j, row start}, {first incidence, incidences, row length, 0}
__device__ __forceinline__ void fin_pack_one(int u, int m, int kg, const int *__restrict__ up_list,
                                             const int *__restrict__ brow, const int *__restrict__ col,
                                             const int *__restrict__ tpos, const int *__restrict__ row_ptr,
                                             const int *__restrict__ inc_start, const int *__restrict__ nbr,
                                             int4 *__restrict__ info, const int *s_base, int *bin_fill, int nu,
                                             int *__restrict__ status)
{
    const int b = up_list[u];
    const int j = brow[b], l = col[b];
    const int i0 = inc_start[b], ni = inc_start[b + 1] - i0;
    if (j == l) {
        const int rp0 = row_ptr[j], len = row_ptr[j + 1] - rp0;
        info[2 * u] = make_int4(b, j, l, rp0);
        info[2 * u + 1] = make_int4(i0, ni, len, 0);
    } else {
        int flags = 0;
        for (int s = 0; s < kg; ++s) {
            if (nbr[j * kg + s] == l) flags |= 1;
            if (nbr[l * kg + s] == j) flags |= 2;
        }
        // off-diagonal records in decreasing order of their incidence counts
        // (the assembly pairs neighbouring records on one warp and starts the
        // long ones first; a block's sums do not depend on its slot)
        const int bin = ni < ED_ASM_BINS - 1 ? ni : ED_ASM_BINS - 1;
        const int d = m + s_base[bin] + atomicAdd(&bin_fill[bin], 1);
        if (d >= nu) {   // (the classes count the same strictly upper blocks: never)
            atomicCAS(status, ED_OK, ED_ERR_STATE);
            return;
        }
        info[2 * d] = make_int4(b, j, l, tpos[b]);
        info[2 * d + 1] = make_int4(i0, ni, flags, 0);
    }
}


__global__ void k_fin_pack(const int *__restrict__ nnzb_dev, int cap, int m, int kg, const int *__restrict__ up_list,
                           const int *__restrict__ flag_b, const int *__restrict__ brow, const int *__restrict__ col,
                           const int *__restrict__ tpos, const int *__restrict__ row_ptr,
                           const int *__restrict__ inc_start, const int *__restrict__ nbr, int4 *__restrict__ info,
                           int *__restrict__ bins, int *__restrict__ status)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    // first slot of every incidence-count class, largest class first
    __shared__ int s_base[ED_ASM_BINS];
    if (threadIdx.x < ED_ASM_BINS) {
        int sum = 0;
        for (int q = ED_ASM_BINS - 1; q > (int)threadIdx.x; --q) sum += bins[q];
        s_base[threadIdx.x] = sum;
    }
    __syncthreads();
    const int nnzb = *nnzb_dev;
    if (nnzb > cap) return;
    const int nu = m + flag_b[nnzb];   // the upper-block count
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x)
        fin_pack_one(u, m, kg, up_list, brow, col, tpos, row_ptr, inc_start, nbr, info, s_base, bins + ED_ASM_BINS, nu,
                     status);
}


// ---------------------------------------------------------------------------

// the three rows of every key point after the model points
__global__ void k_kp_expand(const float4 *__restrict__ kp, int nk, int n_model, float4 *__restrict__ pos,
                            float4 *__restrict__ nrm)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nk) return;
    const float4 p = kp[t / 3];
    pos[n_model + t] = make_float4(p.x, p.y, p.z, 0.f);
    nrm[n_model + t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// node counts of the sampled graph: counts[0] = min(sampled, max_nodes), counts[1] = sampled
// (and the count in use to misc[MI_M], which goes to the host with the other misc words)
__global__ void k_set_counts(int *__restrict__ misc, int max_nodes, int *__restrict__ counts)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int mt = misc[MI_PHASE_BASE];
    const int mu = mt < max_nodes ? mt : max_nodes;
    counts[0] = mu;
    counts[1] = mt;
    misc[MI_M] = mu;
}

// the block count into the graph's counts[2] (counts[3] = 0)
__global__ void k_counts_pattern(const int *__restrict__ misc, int *__restrict__ counts)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    counts[2] = misc[MI_READ];
    counts[3] = 0;
}

// bounding box of n points into misc[MI_BBOX .. MI_BBOX + 5] (ordered ints)
ed_status ed_bbox_enqueue(ed_context *ctx, const float4 *pos, int n, cudaStream_t st)
{
    k_bbox_init<<<1, 32, 0, st>>>(ctx->misc); ed_note_launch();
    if (n > 0) {
        ED_LAUNCH(k_bbox, min(ed_div_up(n, 256), 4 * ctx->num_sms), 256, st, pos, n, ctx->misc); ed_note_launch();
    }
    ED_LAUNCH_CHECK();
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
    const int N = n_points;                     // model points: the bounding box and the nodes
    const int NT = n_points + 3 * ctx->n_kp;    // model points and key-point rows: skinning, pattern, entries
    if (NT > ctx->lim.max_points) return ED_ERR_CAPACITY;
    const float4 *P4 = (const float4 *)pos;
    const float4 *PT = P4;                      // the extended point set
    if (ctx->n_kp > 0) {
        ED_CUDA_TRY(cudaMemcpyAsync(ctx->comb_pos, pos, sizeof(float4) * (size_t)N, cudaMemcpyDeviceToDevice, st));
        ED_CUDA_TRY(cudaMemcpyAsync(ctx->comb_nrm, nrm, sizeof(float4) * (size_t)N, cudaMemcpyDeviceToDevice, st));
        ED_LAUNCH(k_kp_expand, ed_div_up(3 * ctx->n_kp, 256), 256, st, ctx->kp_pos, ctx->n_kp, N, ctx->comb_pos,
                                                                   ctx->comb_nrm); ed_note_launch();
        PT = ctx->comb_pos;
    }
    float4 *G4 = (float4 *)graph->nodes;
    int hm[MI_COUNT];
    ed_status s;
    // ---- bounding box and grids ----
    ED_LAUNCH(k_build_init, 2 * ctx->num_sms, 256, st, ctx->misc, ctx->bcnt, 2 * (max_nodes + 1), ctx->icnt,
              2 * (ctx->max_nnzb + 1) + 2 * ED_ASM_BINS); ed_note_launch();
    ED_LAUNCH(k_bbox, min(ed_div_up(N, 256), 4 * ctx->num_sms), 256, st, P4, N, ctx->misc); ed_note_launch();
    float kc = prm->search_cell;
    if (!(kc > 0.f)) kc = m_in > 0 ? (prm->sigma > 0.f ? prm->sigma : 1.0f) : 2.0f * prm->node_radius;
    ED_LAUNCH(k_grid_setup, 1, 1, st, ctx->misc, ctx->fmisc, m_in > 0 ? 1.0f : prm->node_radius, kc, ctx->lim.max_cells,
                                  m_in == 0); ed_note_launch();
    ED_LAUNCH_CHECK();
    // the grid dims go to the host without draining the stream
    ED_CUDA_TRY(cudaMemcpyAsync(ctx->misc_host, ctx->misc, sizeof(int) * MI_COUNT, cudaMemcpyDeviceToHost, st));
    ED_CUDA_TRY(cudaEventRecord(ctx->ev_misc, st));

    // ---- nodes: the sampling launches need no host value, so they are queued
    // before the grid dims are waited for (the sampler runs meanwhile); every
    // one of them returns at once when the set-up failed ----
    int m;
    int *pcnt = ctx->misc + MI_PHASES, *pstart = ctx->misc + MI_PHASES + 32, *pfill = ctx->misc + MI_PHASES + 64;
    if (m_in == 0) {
        int2 *bucket = reinterpret_cast<int2 *>(ctx->ent_key);  // N (point, cell) pairs; the entry keys come later
        ED_LAUNCH(k_fill_cells, 4 * ctx->num_sms, 256, st, ctx->cell_pick, ctx->misc); ed_note_launch();
        const int pg = min(ed_div_up(N, 256), 4 * ctx->num_sms);
        ED_LAUNCH(k_cell_of, ed_div_up(N, 256), 256, st, P4, N, ctx->misc, ctx->fmisc, ctx->cell_of); ed_note_launch();
        ED_LAUNCH(k_phase_count, pg, 256, st, ctx->cell_of, N, ctx->misc, pcnt); ed_note_launch();
        ED_LAUNCH(k_phase_scan, 1, 32, st, pcnt, pstart, pfill); ed_note_launch();
        ED_LAUNCH(k_phase_scatter, pg, 256, st, ctx->cell_of, N, ctx->misc, pstart, pfill, bucket); ed_note_launch();
        ED_LAUNCH_CHECK();
        // one cooperative launch for the 27 phases: one CTA per SM (fewer
        // barrier arrivals), sized down for small inputs.  A phase's points are
        // spread over all warps (six per warp and round); the grid is sized for
        // 1.5x the mean points per phase, since phases hold up to ~10% more than
        // the mean and one sized for the mean takes two rounds on those phases
        static int per_sm = -1;   // resident sampler CTAs per SM (the same for every call)
        if (per_sm < 0) ED_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_poisson_all, POISSON_T, 0));
        int pick_grid = min(ed_div_up((N / 18 + 1) * 32 / 6 + 32, POISSON_T), min(per_sm, 1) * ctx->num_sms);
        if (pick_grid < 1) pick_grid = 1;
        {   // the arrival counter was cleared with the misc words above
            const int *misc_c = ctx->misc, *pstart_c = pstart;
            const float *fmisc_c = ctx->fmisc;
            const int2 *bucket_c = bucket;
            int *cell_pick = ctx->cell_pick;
            unsigned *bar = (unsigned *)(ctx->misc + MI_BAR_GRAPH);
            int *status = ctx->misc + MI_STATUS;
            unsigned long long wait_ns = ctx->wait_ns;
            void *args[] = {(void *)&P4, (void *)&bucket_c, (void *)&pstart_c, (void *)&misc_c, (void *)&fmisc_c,
                            (void *)&cell_pick, (void *)&bar, (void *)&status, (void *)&wait_ns};
            ed_note_launch();
            ED_CUDA_TRY(ed_launch_coop((const void *)k_poisson_all, pick_grid, POISSON_T, args, 0, st, true));
        }
    }
    ED_CUDA_TRY(cudaEventSynchronize(ctx->ev_misc));
    memcpy(hm, ctx->misc_host, sizeof(int) * MI_COUNT);
    if (hm[MI_STATUS] != ED_OK) return (ed_status)hm[MI_STATUS];
    if (m_in == 0) {
        // node numbers in (phase, cell) order
        PhaseTable T;
        const int dx = hm[MI_DIMS], dy = hm[MI_DIMS + 1], dz = hm[MI_DIMS + 2];
        int tot = 0;
        for (int ph = 0; ph < 27; ++ph) {
            const int px = ph % 3, py = (ph / 3) % 3, pz = ph / 9;
            T.ax[ph] = dx > px ? (dx - px + 2) / 3 : 0;
            T.ay[ph] = dy > py ? (dy - py + 2) / 3 : 0;
            const int az = dz > pz ? (dz - pz + 2) / 3 : 0;
            T.off[ph] = tot;
            tot += T.ax[ph] * T.ay[ph] * az;
        }
        T.off[27] = tot;
        int *flags = ctx->cell_node, *pre = ctx->kcell_start;   // cells (+ 1) ints each
        ED_LAUNCH(k_node_flags, ed_div_up(tot, 256), 256, st, T, tot, ctx->misc, ctx->cell_pick, flags); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, flags, pre, tot, st, ctx->misc + MI_PHASE_BASE)) != ED_OK) return s;
        ED_LAUNCH(k_node_write, ed_div_up(tot, 256), 256, st, T, tot, ctx->misc, ctx->cell_pick, pre, P4, G4, max_nodes); ed_note_launch();
        ED_LAUNCH_CHECK();
        ED_LAUNCH(k_set_counts, 1, 1, st, ctx->misc, max_nodes, graph->counts); ed_note_launch();
    } else {
        ctx->pinned[ED_MAX_PCG_GRID + 3] = m_in;
        ctx->pinned[ED_MAX_PCG_GRID + 4] = m_in;
        ED_CUDA_TRY(cudaMemcpyAsync(graph->counts, ctx->pinned + ED_MAX_PCG_GRID + 3, 2 * sizeof(int),
                                    cudaMemcpyHostToDevice, st));
    }
    // the node count goes to the host while the next kernels run: they read it
    // from graph->counts and are sized for max_nodes
    ED_CUDA_TRY(cudaMemcpyAsync(ctx->misc_host, ctx->misc, sizeof(int) * MI_COUNT, cudaMemcpyDeviceToHost, st));
    ED_CUDA_TRY(cudaEventRecord(ctx->ev_misc, st));

    // ---- node graph on the context's second stream (it needs only the nodes;
    // only the block pattern reads it), beside the nearest nodes and weights ----
    const int *m_dev = graph->counts;
    ED_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
    ED_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    k_node_graph<<<ed_div_up(max_nodes, NG_WARPS), 32 * NG_WARPS, 0, ctx->aux>>>(G4, m_dev, prm->k_graph, graph->nbr, ctx->bitmap,
                                                                                   max_nodes * ed_div_up(max_nodes, 32)); ed_note_launch();
    ED_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->aux));
    {
        const int kcells = hm[MI_KDIMS + 3];
        ED_CUDA_TRY(cudaMemsetAsync(ctx->kcell_cnt, 0, sizeof(int) * (kcells + 1), st));
        int *cell_of_node = ctx->row_cnt;   // scratch (m + 1 ints)
        ED_LAUNCH(k_kcell_count, ed_div_up(max_nodes, 256), 256, st, G4, m_dev, ctx->misc, ctx->fmisc, ctx->kcell_cnt,
                                                                 cell_of_node); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->kcell_cnt, ctx->kcell_start, kcells, st)) != ED_OK) return s;
        ED_LAUNCH(k_kcell_fill, ed_div_up(max_nodes, 256), 256, st, m_dev, G4, ctx->kcell_start, ctx->kcell_cnt,
                                                                cell_of_node, ctx->kcell_pos); ed_note_launch();
        ED_LAUNCH(k_knn, ed_div_up(NT, 128), 128, st, PT, NT, G4, m_dev, ctx->misc, ctx->fmisc, ctx->kcell_start,
                                                  ctx->kcell_pos, prm->weight_mode, prm->sigma,
                                                  (ushort4 *)graph->idx, (float4 *)graph->weights); ed_note_launch();
        ED_LAUNCH_CHECK();
    }
    // ---- the points sorted by their node tuple, and the runs of equal tuples
    // (queued before the node count is waited for: they need only the nearest
    // nodes; the number of runs goes to the host with the block count) ----
    {
        int fb = 1;
        while ((1 << fb) < max_nodes) ++fb;
        const ushort4 *I4 = (const ushort4 *)graph->idx;
        if ((long)NT <= 512L * max_nodes) {
            // buckets by smallest node (a few hundred points each at the node
            // densities of the path), each ordered by ranks
            // (bcnt and its fill counters were zeroed by k_build_init)
            int *bfill = ctx->bcnt + max_nodes + 1;
            ED_LAUNCH(k_tb_count, ed_div_up(NT, 256), 256, st, I4, NT, ctx->bcnt); ed_note_launch();
            ED_LAUNCH_CHECK();
            if ((s = ed_scan_exclusive(ctx, ctx->bcnt, ctx->bstart, max_nodes, st)) != ED_OK) return s;
            ED_LAUNCH(k_tb_place, ed_div_up(NT, 256), 256, st, I4, NT, ctx->bstart, bfill, ctx->ent_key); ed_note_launch();
            int pb = 1;
            while ((1L << pb) < (long)NT) ++pb;
            if (3 * fb + pb <= 64) {
                ED_LAUNCH(k_tb_sort64, max_nodes, TB64_T, st, I4, ctx->bstart, max_nodes, fb, pb, ctx->ent_key, ctx->ent_val); ed_note_launch();
            } else {
                ED_LAUNCH(k_tb_sort, max_nodes, TB_T, st, I4, ctx->bstart, max_nodes, fb, ctx->ent_key, ctx->ent_val); ed_note_launch();
            }
            ED_LAUNCH_CHECK();
        } else {
            // few nodes for many points: large buckets; a stable radix sort by the full key
            ED_LAUNCH(k_tuple_lo, ed_div_up(NT, 256), 256, st, I4, NT, fb, ctx->ent_key, ctx->ent_val); ed_note_launch();
            ED_LAUNCH_CHECK();
            if ((s = ed_radix_sort_pairs(ctx, ctx->ent_key, ctx->ent_val, NT, 4 * fb < 32 ? 4 * fb : 32, st)) != ED_OK)
                return s;
            if (4 * fb > 32) {
                k_tuple_hi<<<ed_div_up(NT, 256), 256, 0, st>>>(I4, NT, fb, ctx->ent_val, ctx->ent_key); ed_note_launch();
                ED_LAUNCH_CHECK();
                if ((s = ed_radix_sort_pairs(ctx, ctx->ent_key, ctx->ent_val, NT, 4 * fb - 32, st)) != ED_OK) return s;
            }
        }
        const float4 *NR = ctx->n_kp > 0 ? (const float4 *)ctx->comb_nrm : (const float4 *)nrm;
        ED_LAUNCH(k_tuple_gather, ed_div_up(NT, 256), 256, st, ctx->ent_val, NT, I4, (const float4 *)graph->weights, PT, NR,
                                                           ctx->perm, ctx->spos, ctx->snrm, ctx->sidx, ctx->sw,
                                                           ctx->sidx_d, ctx->sw_d, ctx->flag_a); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->flag_a, ctx->flag_b, NT, st, ctx->misc + MI_READ + 1)) != ED_OK) return s;
        ED_LAUNCH(k_run_starts, ed_div_up(NT, 256), 256, st, ctx->flag_a, ctx->flag_b, NT, ctx->run_start,
                                                         ctx->run_of_start); ed_note_launch();
        ED_LAUNCH_CHECK();
    }
    // every later launch on the caller's stream (and every return) follows the node graph
    ED_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    ED_CUDA_TRY(cudaEventSynchronize(ctx->ev_misc));
    memcpy(hm, ctx->misc_host, sizeof(int) * MI_COUNT);
    if (hm[MI_STATUS] != ED_OK) return (ed_status)hm[MI_STATUS];
    m = m_in > 0 ? m_in : hm[MI_M];
    if (m < ED_K || (prm->weight_mode == ED_WEIGHT_EQ2 && m < ED_K + 1) || m <= prm->k_graph) return ED_ERR_ARG;

    // ---- block pattern ----
    const int words = ed_div_up(m, 32);
    const int cap = ctx->max_nnzb;
    const int *nnzb_dev = ctx->misc + MI_READ, *nruns_dev = ctx->misc + MI_READ + 1;
    const int g256 = 4 * ctx->num_sms;   // grid of the grid-stride launches over blocks and runs
    {
        // (the bitmap was zeroed by k_node_graph: m x words <= max_nodes x words(max_nodes))
        // (the pairs of the points come from their runs: n_runs is on the device, the
        // grid covers every point)
        k_pairs_runs_dev<<<ed_div_up(NT, 256), 256, 0, st>>>(ctx->misc + MI_READ + 1, ctx->run_start, ctx->sidx,
                                                             ctx->bitmap, words); ed_note_launch();
        ED_LAUNCH(k_pairs_graph, ed_div_up(m, 256), 256, st, graph->nbr, m, prm->k_graph, ctx->bitmap, words); ed_note_launch();
        ED_LAUNCH(k_row_count, ed_div_up(m, 4), 128, st, ctx->bitmap, m, words, ctx->row_cnt); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->row_cnt, ctx->row_ptr, m, st, ctx->misc + MI_READ)) != ED_OK) return s;
        // the block count and the number of runs go to the host (pinned copy +
        // event) while the block lists, which need only the row pointer, are
        // filled (checking the count against the capacity)
        ED_LAUNCH(k_row_fill, ed_div_up(m, 4), 128, st, ctx->bitmap, m, words, ctx->row_ptr, ctx->col, ctx->brow,
                                                    ctx->diag_pos, ctx->max_nnzb, ctx->misc + MI_STATUS); ed_note_launch();
        ED_LAUNCH_CHECK();
        // from here on the block count (misc[MI_READ]) and the run count
        // (misc[MI_READ + 1]) are read on the device: the launches are sized
        // for the capacities, grid-stride, and nothing runs past a block count
        // above the capacity (the row fill reported ED_ERR_CAPACITY)
        ED_LAUNCH(k_tpos, g256, 256, st, nnzb_dev, cap, ctx->row_ptr, ctx->col, ctx->brow, ctx->tpos, ctx->flag_a); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->flag_a, ctx->flag_b, cap, st, ctx->misc + MI_READ + 2, nnzb_dev)) != ED_OK)
            return s;
        ED_LAUNCH(k_compact_upper, g256, 256, st, nnzb_dev, cap, m, ctx->flag_a, ctx->flag_b, ctx->diag_pos, ctx->up_list); ed_note_launch();
        ED_LAUNCH_CHECK();
    }

    // ---- incidences (block, run), sorted by block (stable: run order within a
    // block), and the assembly's per-block records ----
    {
        ED_LAUNCH(k_inc_gen, g256, 256, st, nruns_dev, nnzb_dev, cap, ctx->run_start, ctx->sidx, ctx->row_ptr, ctx->col,
                                        ctx->ent_key, ctx->ent_val, ctx->misc + MI_STATUS); ed_note_launch();
        ED_LAUNCH_CHECK();
        // by block, each block's list in run order
        // (icnt and its fill counters were zeroed by k_build_init)
        int *ifill = ctx->icnt + cap + 1;
        ED_LAUNCH(k_ic_count, 4 * g256, 256, st, nruns_dev, nnzb_dev, cap, ctx->ent_key, ctx->icnt); ed_note_launch();
        ED_LAUNCH_CHECK();
        if ((s = ed_scan_exclusive(ctx, ctx->icnt, ctx->ent_start, cap, st, nullptr, nnzb_dev)) != ED_OK) return s;
        ED_LAUNCH(k_ic_place, 4 * g256, 256, st, nruns_dev, nnzb_dev, cap, ctx->ent_key, ctx->ent_val, ctx->ent_start,
                                              ifill, ctx->inc); ed_note_launch();
        ED_LAUNCH(k_ic_sort, std::min(ed_div_up(cap, 4), 32 * ctx->num_sms), 128, st, nnzb_dev, cap, ctx->ent_start,
                  ctx->inc, ctx->brow, ctx->col, ctx->asm_bins); ed_note_launch();
        ED_LAUNCH(k_fin_pack, g256, 256, st, nnzb_dev, cap, m, prm->k_graph, ctx->up_list, ctx->flag_b, ctx->brow, ctx->col,
                                         ctx->tpos, ctx->row_ptr, ctx->ent_start, graph->nbr, ctx->fin_info, ctx->asm_bins,
                                         ctx->misc + MI_STATUS); ed_note_launch();
        ED_LAUNCH(k_counts_pattern, 1, 1, st, ctx->misc, graph->counts); ed_note_launch();
        ED_LAUNCH_CHECK();
        // what the host needs later (the counts, the row pointer of the PCG
        // plan) goes to pinned memory; ed_graph_ready reads it at the first
        // call that needs it
        ED_CUDA_TRY(cudaMemcpyAsync(ctx->row_ptr_host, ctx->row_ptr, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost, st));
        ED_CUDA_TRY(cudaMemcpyAsync(ctx->misc_host, ctx->misc, sizeof(int) * MI_COUNT, cudaMemcpyDeviceToHost, st));
        ED_CUDA_TRY(cudaEventRecord(ctx->ev_build, st));
    }

    ctx->pos = ctx->n_kp > 0 ? (const float *)ctx->comb_pos : pos;
    ctx->nrm = ctx->n_kp > 0 ? (const float *)ctx->comb_nrm : nrm;
    ctx->N = NT;
    ctx->n_model = N;
    ctx->graph = *graph;
    ctx->k_graph = prm->k_graph;
    ctx->weight_mode = prm->weight_mode;
    ctx->sigma = prm->sigma;
    ctx->m = m;
    ctx->n_entries = 10 * NT;
    ctx->build_pending = 1;
    ctx->have_graph = 1;
    return ED_OK;
}

// The pattern's counts and the PCG plan of the last build, once its queued
// work has reached the copies of ed_build_graph's end (one host wait, at the
// first call that needs them).  An error the build's kernels reported is
// returned here, and the context then has no graph.
ed_status ed_graph_ready(ed_context *ctx, cudaStream_t st)
{
    if (!ctx->have_graph) return ED_ERR_STATE;
    if (!ctx->build_pending) return ED_OK;
    ctx->build_pending = 0;
    ctx->have_graph = 0;
    ED_CUDA_TRY(cudaEventSynchronize(ctx->ev_build));
    int hm[MI_COUNT];
    memcpy(hm, ctx->misc_host, sizeof(int) * MI_COUNT);
    if (hm[MI_STATUS] != ED_OK) return (ed_status)hm[MI_STATUS];
    const int m = ctx->m, nnzb = hm[MI_READ], n_runs = hm[MI_READ + 1], n_upper = hm[MI_READ + 2] + m;
    if (nnzb > ctx->max_nnzb) return ED_ERR_CAPACITY;
    if (n_runs < 1 || n_runs > ctx->N) return ED_ERR_STATE;
    if (2 * n_upper != nnzb + m) return ED_ERR_STATE;   // the pattern must be symmetric with a full diagonal
    ctx->nnzb = nnzb;
    ctx->n_upper = n_upper;
    ctx->n_runs = n_runs;
    // row partition and shared-memory plan of the PCG solve
    ed_status s = ed_pcg_plan(ctx, ctx->row_ptr_host, st);
    if (s != ED_OK) return s;
    ctx->have_graph = 1;
    return ED_OK;
}
