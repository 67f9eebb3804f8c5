// pcg.cu -- block-Jacobi preconditioned conjugate gradients on the normal
// equations of one Gauss-Newton step (Sec. II.F), as one persistent
// cooperative kernel.
//
// H is a symmetric block-sparse matrix over the m nodes (12x12 blocks, both
// triangles stored, row-major blocks) bordered by the 6 pose unknowns:
// pose-node blocks C_j (6x12) and a 6x6 pose block.  Each CTA (one per SM)
// owns a contiguous range of node rows, balanced by block count at graph
// build.  For the whole solve a CTA keeps in shared memory its rows' blocks
// (as many as fit; the rest stream from L2), block inverses, pose-node
// blocks, its slices of d, r, z, p, q, s and the z and p of every block
// column its rows touch; the pose parts of the vectors are kept, identical,
// in every CTA.
//
// One grid barrier per iteration.  After q = H p a CTA forms s = M^-1 q for
// its rows and publishes it, together with its partials of p.q, q.z, q.s,
// r.z, r.r, r.q, q.q and C p; after the barrier every CTA has the sums,
// alpha = r.z / p.q, and beta from r'.z' = r.z - 2 alpha q.z + alpha^2 q.s
// (z' = z - alpha s), and updates its block columns' z and p from the
// owners' s exactly as the owners do (same fused multiply-adds, so every
// copy agrees bit for bit).  r.z itself is summed afresh at every barrier,
// so alpha never rests on the recurrence.  In exact arithmetic this is the
// standard preconditioned CG.  Reductions are per-CTA partials summed in a
// fixed order by every CTA: deterministic.
#include <mutex>

#include "ed_internal.cuh"

#define PCG_SMEM_MAX (200 * 1024)      // one 512-thread CTA per SM
#define PCG_SMEM_MAX_256 (100 * 1024)  // two 256-thread CTAs per SM

#define PCG_RI 2                       // staged column items per thread held in registers
#define PCG_NC 13                      // partials per CTA and iteration: p.q, q.z, q.s, r.z, r.r, r.q, q.q, C p

// 12 threads per node row (one per output row of a 12x12 block)
template <int NT> struct RowsPerPass { static constexpr int v = NT / 12; };

struct PcgArgs {
    int m, n_iter;
    float tol;
    const int *row_ptr, *col;
    const int *cta_rows;     // [grid + 1] first row of every CTA
    int n_cache;             // blocks of each CTA cached in shared memory
    int max_rows, max_blk;   // shared-memory plan
    const float *bsr, *pnode, *minv, *pose_blk, *grad;
    float *d;                // the solution
    float *s0, *s1;          // published s = M^-1 q of even / odd iterations
    double *part;            // [2][PCG_NC][ED_MAX_PCG_GRID] partials of even / odd iterations, component-major
                             // (stored in the accumulator's type: float in FP32 mode, float2 in mixed mode)
    float *x;                // node parameters, x += d at the end (all CTAs passed every barrier)
    double *xm;              // FP64 master copy (mixed precision) or NULL
    double *pose;            // pose += d_pose (CTA 0)
    int load_before_wait;    // 1: the set-up's loads come before the wait for the stream predecessor (which
                             // then must be k_fin_totals: everything these loads read is two kernels back)
    unsigned *bar;           // arrival count
    unsigned bar_extra;      // arrivals expected beyond the CTAs (0; > 0 only in tests of the bounded wait)
    unsigned long long wait_ns;   // limit of every device wait
    int *status;
    ed_stats *stats;
};

// Accumulation of the PCG dot products and norms.  FP32 mode: float.  Mixed
// FP64 mode: double.  Mixed mode: float-float (hi + lo, about 44 significant
// bits) on the FP32 pipe --
// each product is formed exactly (a b = p + e with e = fma(a, b, -p)) and
// summed by error-free two-sums; on B300 the FP64 rate is a small fraction of
// the FP32 rate, so the extended precision is kept off the FP64 units (the
// per-CTA partials between CTAs are stored in the accumulator's own type:
// a conversion to and from double would run on those units).
template <typename DT> struct PcgAcc;

template <> struct PcgAcc<float> {
    typedef float T;
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ T madd(T acc, float a, float b) { return acc + a * b; }
    static __device__ __forceinline__ T add(T x, T y) { return x + y; }
    static __device__ __forceinline__ T shfl(T x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
    static __device__ __forceinline__ T shfl_down(T x, int o) { return __shfl_down_sync(0xffffffffu, x, o); }
    static __device__ __forceinline__ float to_float(T x) { return x; }
};

// FP64 accumulation (ED_PRECISION_MIXED_FP64): products and sums in double
struct PcgFp64 {};
template <> struct PcgAcc<PcgFp64> {
    typedef double T;
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T madd(T acc, float a, float b) { return fma((double)a, (double)b, acc); }
    static __device__ __forceinline__ T add(T x, T y) { return x + y; }
    static __device__ __forceinline__ T shfl(T x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
    static __device__ __forceinline__ T shfl_down(T x, int o) { return __shfl_down_sync(0xffffffffu, x, o); }
    static __device__ __forceinline__ float to_float(T x) { return (float)x; }
};

template <> struct PcgAcc<double> {
    typedef float2 T;
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ T madd(T acc, float a, float b)
    {
        const float p = __fmul_rn(a, b);
        return ed_ff_add(acc, make_float2(p, __fmaf_rn(a, b, -p)));
    }
    static __device__ __forceinline__ T add(T x, T y) { return ed_ff_add(x, y); }
    static __device__ __forceinline__ T shfl(T x, int o)
    {
        return make_float2(__shfl_xor_sync(0xffffffffu, x.x, o), __shfl_xor_sync(0xffffffffu, x.y, o));
    }
    static __device__ __forceinline__ T shfl_down(T x, int o)
    {
        return make_float2(__shfl_down_sync(0xffffffffu, x.x, o), __shfl_down_sync(0xffffffffu, x.y, o));
    }
    static __device__ __forceinline__ float to_float(T x) { return x.x + x.y; }
};

// component w of the partials of CTA c
template <typename DT>
__device__ __forceinline__ typename PcgAcc<DT>::T *part_at(double *part, int w, int c)
{
    return reinterpret_cast<typename PcgAcc<DT>::T *>(part) + (size_t)w * ED_MAX_PCG_GRID + c;
}

// work split of the sum of NC partial components over the warps of a CTA:
// WPC warps per component (all warps when NC is small) stride over the CTAs,
// components in rounds of GROUPS when there are more components than warps
template <int NT, int NC> struct PartSplit {
    static constexpr int NWARP = NT / 32;
    static constexpr int WPC = NWARP >= NC ? NWARP / NC : 1;
    static constexpr int GROUPS = NWARP / WPC;
    static constexpr int ROUNDS = (NC + GROUPS - 1) / GROUPS;
    static_assert(ROUNDS <= 8, "warp results of one component round per sh column");
};

// first stage of the sum of the NC components of all CTA partials: every
// warp's share through a fixed shuffle tree into `sh`, then one CTA barrier.
// Components whose bit is set in `skip` are not loaded (their totals read 0).
// sum_partials_get gives the totals (a fixed-order sum of the warp results,
// the same in every CTA and thread).  `sh` must not be in use by other code
// between the two.
template <typename DT, int NT, int NC>
__device__ __forceinline__ void sum_partials(double *part, int nb, typename PcgAcc<DT>::T (*sh)[8], unsigned skip = 0u)
{
    typedef PcgAcc<DT> A;
    typedef PartSplit<NT, NC> S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = wid / S::WPC, wsub = wid - g * S::WPC;
#pragma unroll
    for (int rd = 0; rd < S::ROUNDS; ++rd) {
        const int c = rd * S::GROUPS + g;
        typename A::T s = A::zero();
        if (g < S::GROUPS && c < NC && !((skip >> c) & 1u)) {
            const typename A::T *src = part_at<DT>(part, c, 0);
            // every load of the lane in flight before the first add (up to 8 per lane)
            typename A::T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = wsub * 32 + lane + u * S::WPC * 32;
                v[u] = k < nb ? __ldcg(src + k) : A::zero();
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (wsub * 32 + lane + u * S::WPC * 32 < nb) s = A::add(s, v[u]);
            for (int k = wsub * 32 + lane + 8 * S::WPC * 32; k < nb; k += S::WPC * 32)
                s = A::add(s, __ldcg(src + k));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl(s, o));
        if (lane == 0) sh[wid][rd] = s;
    }
    __syncthreads();
}

template <typename DT, int NT, int NC>
__device__ __forceinline__ typename PcgAcc<DT>::T sum_partials_get(const typename PcgAcc<DT>::T (*sh)[8], int c)
{
    typedef PcgAcc<DT> A;
    typedef PartSplit<NT, NC> S;
    const int rd = c / S::GROUPS, gg = c - rd * S::GROUPS;
    typename A::T r = A::zero();
#pragma unroll
    for (int k = 0; k < S::WPC; ++k) r = A::add(r, sh[gg * S::WPC + k][rd]);
    return r;
}

// block reduction of NV values per thread: after one CTA barrier,
// block_sum_get(c) gives component c (fixed order) to any thread that asks
template <typename DT, int NT, int NV, int SW>
__device__ __forceinline__ void block_sum_n(typename PcgAcc<DT>::T (&v)[NV], typename PcgAcc<DT>::T (*sh)[SW])
{
    typedef PcgAcc<DT> A;
    static_assert(NV <= SW, "one shared column per value");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        typename A::T x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = A::add(x, A::shfl(x, o));
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
}

// the same for several values: a butterfly over the warp that halves the
// values a lane carries at every step (lane bit o keeps the upper or the lower
// half and receives that half from its partner), so lanes 2c and 2c + 1 end
// with value c's warp total -- about 2 NV shuffles instead of 5 NV
template <typename DT, int NT, int NV, int SW>
__device__ __forceinline__ void block_sum_bfly(const typename PcgAcc<DT>::T (&v)[NV], typename PcgAcc<DT>::T (*sh)[SW])
{
    typedef PcgAcc<DT> A;
    typedef typename A::T T;
    static_assert(NV > 1 && NV <= 16 && NV <= SW, "up to 16 values, one shared column each");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = k < NV ? v[k] : A::zero();
#pragma unroll
    for (int lvl = 0; lvl < 4; ++lvl) {
        const int o = 16 >> lvl, half = 8 >> lvl;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const T send = up ? x[j] : x[j + half];
            const T keep = up ? x[j + half] : x[j];
            x[j] = A::add(keep, A::shfl(send, o));
        }
    }
    const T r = A::add(x[0], A::shfl(x[0], 1));
    const int c = lane >> 1;
    if (!(lane & 1) && c < NV) sh[wid][c] = r;
    __syncthreads();
}

template <typename DT, int NT, int SW>
__device__ __forceinline__ typename PcgAcc<DT>::T block_sum_get(const typename PcgAcc<DT>::T (*sh)[SW], int c)
{
    typedef PcgAcc<DT> A;
    typename A::T s = A::zero();
    for (int w = 0; w < NT / 32; ++w) s = A::add(s, sh[w][c]);
    return s;
}

// shared-memory carve of one CTA (in floats; every region a multiple of 4)
struct PcgSmem {
    size_t o_H, o_pb, o_po, o_lc, o_M, o_C, o_r, o_d, o_z, o_p, o_q, o_s, o_qs, total;
};

__host__ __device__ inline PcgSmem pcg_smem_layout(int rows, int nblk, int ncache, int nt)
{
    PcgSmem L;
    size_t o = 0;
    L.o_H = o; o += (size_t)ncache * 144;
    L.o_pb = o; o += (size_t)nblk * 12;            // p of the block columns
    L.o_po = o; o += (size_t)nblk * 12;            // z of the block columns
    L.o_lc = o; o += ((size_t)nblk + 3) / 4 * 4;   // block column indices (int)
    L.o_M = o; o += (size_t)rows * 144;
    L.o_C = o; o += (size_t)rows * 72;
    L.o_r = o; o += (size_t)rows * 12;
    L.o_d = o; o += (size_t)rows * 12;
    L.o_z = o; o += (size_t)rows * 12;
    L.o_p = o; o += (size_t)rows * 12;
    L.o_q = o; o += (size_t)rows * 12;
    L.o_s = o; o += (size_t)rows * 12;
    L.o_qs = o; o += (size_t)(nt / 12) * 12;       // split partial products of q
    L.total = o;
    return L;
}

// a row of a 12x12 block times a 12-vector, rounded in a fixed order: a CTA
// forms z = M^-1 r for its own rows and, from the owners' data, for the copies
// of its block columns, and the copies must agree with the owners bit for bit
__device__ __forceinline__ float dot12(const float4 (&m)[3], const float4 (&v)[3])
{
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float d = __fmul_rn(m[q].x, v[q].x);
        d = __fmaf_rn(m[q].y, v[q].y, d);
        d = __fmaf_rn(m[q].z, v[q].z, d);
        d = __fmaf_rn(m[q].w, v[q].w, d);
        acc = __fadd_rn(acc, d);
    }
    return acc;
}

// the solve of one problem by CTA `cta` of the `nb` CTAs given to it
template <typename DT, int NT>
__device__ __forceinline__ void pcg_body(const PcgArgs &a, const int cta, const unsigned nb)
{
    constexpr int ROWS_PER_PASS = RowsPerPass<NT>::v;
    typedef PcgAcc<DT> A;
    typedef typename A::T AT;   // accumulator of the dot products and norms
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ int s_flag;
    __shared__ AT s_red[NT / 32][PCG_NC];   // block reductions
    __shared__ AT s_red2[NT / 32][8];       // sums of the CTA partials
    // the pose parts of r, z, p, d: the same values in every CTA
    __shared__ float s_rp[6], s_zp[6], s_pp[6], s_dp[6];
    __shared__ float s_Hpp[36], s_Mp[36];
    __shared__ float s_hp[6];               // H_pp p_pose of the iteration (formed at its start)
    __shared__ float s_ab[2];               // alpha, beta of the iteration
    __shared__ int s_ctl;                   // 0 go on, 1 converged or stalled, 2 breakdown

    unsigned target = 0;
    const int m = a.m;
    const int r0 = a.cta_rows[cta], r1 = a.cta_rows[cta + 1];
    const int rows = r1 - r0;
    const int b0 = a.row_ptr[r0], nblk = a.row_ptr[r1] - b0;
    const int ncache = min(nblk, a.n_cache);
    const PcgSmem L = pcg_smem_layout(a.max_rows, a.max_blk, a.n_cache, NT);
    float *Hs = sm + L.o_H, *pb = sm + L.o_pb, *zb = sm + L.o_po, *Ms = sm + L.o_M, *Cs = sm + L.o_C;
    float *rs = sm + L.o_r, *ds = sm + L.o_d, *zs = sm + L.o_z, *ps = sm + L.o_p, *qs = sm + L.o_q;
    float *ss = sm + L.o_s, *qsplit = sm + L.o_qs;
    int *lc = reinterpret_cast<int *>(sm + L.o_lc);
    const int t = threadIdx.x;
    const int grp = t / 12, rr = t % 12;
    const bool in_grp = grp < ROWS_PER_PASS;
    // q = H p.  Up to ROWS_PER_PASS rows: every row gets groups of 12 threads
    // in proportion to its blocks (at most T blocks per thread, T as small as
    // the groups allow), mapped here; more rows: one group per row, in passes.
    constexpr int NG = ROWS_PER_PASS;
    const bool split_rows = rows <= NG;
    __shared__ short s_grow[NG], s_gsp[NG];     // group -> row, split index (row -1: idle)
    __shared__ short s_rfirst[NG], s_rcnt[NG];  // row -> first group, groups
    const int P = 12 * m;
    const float *Hpp = s_Hpp, *Mp = s_Mp;

    // a failed solve leaves x and the pose untouched; CTA 0 reports the status
    auto fail = [&]() {
        if (cta == 0 && t == 0 && a.stats) a.stats->status = *(volatile int *)a.status;
    };

    // ---- the CTA's share of H, M^-1 and C into shared memory by bulk
    // asynchronous copies (inverses and pose-node blocks on mbarrier 0, needed
    // first; blocks on mbarrier 1, needed by the first q = H p); block columns,
    // b and z = M^-1 b of the block columns by plain loads meanwhile.  All of it
    // is in bounds whatever the status word says; the status is checked once
    // the copies have landed ----
    __shared__ __align__(8) unsigned long long s_mbar[2];
    if (t == 0) {
        ed_mbar_init(&s_mbar[0], 1);
        ed_mbar_init(&s_mbar[1], 1);
    }
    __syncthreads();
    if (t == 0) {
        const unsigned mbytes = (unsigned)rows * 576u, cbytes = (unsigned)rows * 288u;
        ed_mbar_expect_tx(&s_mbar[0], mbytes + cbytes);
        if (mbytes) ed_bulk_g2s(Ms, a.minv + (size_t)r0 * 144, mbytes, &s_mbar[0]);
        if (cbytes) ed_bulk_g2s(Cs, a.pnode + (size_t)r0 * 72, cbytes, &s_mbar[0]);
        const size_t hbytes = (size_t)ncache * 576;
        ed_mbar_expect_tx(&s_mbar[1], (unsigned)hbytes);
        const char *hsrc = reinterpret_cast<const char *>(a.bsr + (size_t)b0 * 144);
        char *hdst = reinterpret_cast<char *>(Hs);
        for (size_t o = 0; o < hbytes; o += 32768) {
            const unsigned n = (unsigned)(hbytes - o < 32768 ? hbytes - o : 32768);
            ed_bulk_g2s(hdst + o, hsrc + o, n, &s_mbar[1]);
        }
    }
    for (int i = t; i < nblk; i += NT) lc[i] = __ldg(a.col + b0 + i);
    for (int i = t; i < rows * 12; i += NT) {
        rs[i] = -__ldg(a.grad + 12 * r0 + i);
        ds[i] = 0.f;
    }
    if (t < 36) {
        s_Hpp[t] = a.pose_blk[t];
        s_Mp[t] = a.pose_blk[36 + t];
    }
    if (t < 6) {
        s_rp[t] = -__ldg(a.grad + P + t);
        s_dp[t] = 0.f;
    }
    // z = M^-1 r (r = b) and p = z of every block column, formed here from its
    // owner's inverse and gradient with the owner's arithmetic (dot12 on the
    // same values), so no exchange is needed before the first iteration
    for (int i0 = t; i0 < nblk * 12; i0 += 2 * NT) {   // two items per step, their loads together
        float4 m4[2][3], r4[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = i0 + u * NT;
            if (i < nblk * 12) {
                const int lb = i / 12, rw = i - 12 * lb;
                const size_t l = (size_t)__ldg(a.col + b0 + lb);
                const float4 *mv = reinterpret_cast<const float4 *>(a.minv + l * 144 + rw * 12);
                const float4 *gv = reinterpret_cast<const float4 *>(a.grad + 12 * l);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    m4[u][q] = __ldg(mv + q);
                    r4[u][q] = __ldg(gv + q);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = i0 + u * NT;
            if (i < nblk * 12) {
                const int lb = i / 12, rw = i - 12 * lb;
#pragma unroll
                for (int q = 0; q < 3; ++q) r4[u][q] = make_float4(-r4[u][q].x, -r4[u][q].y, -r4[u][q].z, -r4[u][q].w);
                const float z = dot12(m4[u], r4[u]);
                zb[(size_t)lb * 12 + rw] = z;
                pb[(size_t)lb * 12 + rw] = z;
            }
        }
    }
    // (after a wait that gave up, the copies still in flight are waited for
    // with the default limit, which a shortened wait limit does not shorten)
    if (!ed_mbar_wait(&s_mbar[0], 0, a.wait_ns)) {
        atomicCAS(a.status, ED_OK, ED_ERR_TIMEOUT);
        ed_mbar_wait(&s_mbar[0], 0);
        ed_mbar_wait(&s_mbar[1], 0);
        fail();
        return;
    }
    ed_pdl_wait();   // (no-op when it came first or without the launch attribute)
    if (t == 0) s_flag = *(volatile int *)a.status == ED_OK;   // one reading for the whole CTA
    __syncthreads();
    if (!s_flag) {
        ed_mbar_wait(&s_mbar[1], 0);
        fail();
        return;
    }
    bool h_ready = false;
    if (split_rows && t < 32) {   // (read after the CTA barrier at the loop head)
        auto blocks = [&](int j) { return j < rows ? a.row_ptr[r0 + j + 1] - a.row_ptr[r0 + j] : 0; };
        const int bA = blocks(t), bB = blocks(t + 32);
        int T = max(1, (nblk + NG - 1) / NG);
        for (;;) {   // ends: at T = the longest row every row takes one group
            int c = (bA + T - 1) / T + (bB + T - 1) / T;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (c <= NG) break;
            ++T;
        }
        const int gA = (bA + T - 1) / T, gB = (bB + T - 1) / T;
        int xA = gA, xB = gB;   // inclusive scans over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yA = __shfl_up_sync(0xffffffffu, xA, o), yB = __shfl_up_sync(0xffffffffu, xB, o);
            if (t >= o) {
                xA += yA;
                xB += yB;
            }
        }
        const int totA = __shfl_sync(0xffffffffu, xA, 31), tot = totA + __shfl_sync(0xffffffffu, xB, 31);
        if (t < rows) {
            const int f = xA - gA;
            s_rfirst[t] = (short)f;
            s_rcnt[t] = (short)gA;
            for (int q = 0; q < gA; ++q) {
                s_grow[f + q] = (short)t;
                s_gsp[f + q] = (short)q;
            }
        }
        if (t + 32 < rows) {
            const int f = totA + xB - gB;
            s_rfirst[t + 32] = (short)f;
            s_rcnt[t + 32] = (short)gB;
            for (int q = 0; q < gB; ++q) {
                s_grow[f + q] = (short)(t + 32);
                s_gsp[f + q] = (short)q;
            }
        }
        for (int g = tot + t; g < NG; g += 32) s_grow[g] = -1;
    }
    __syncthreads();   // (the group map above, read below)
    // the group's row and block range for q = H p, the same in every iteration
    // (split rows: one pass; otherwise formed per pass in the loop)
    int g_jl = -1, g_sp = 0, g_S = 1, g_bb0 = 0, g_bb1 = 0;
    if (split_rows && in_grp) {
        g_jl = s_grow[grp];
        g_sp = s_gsp[grp];
        g_S = g_jl >= 0 ? s_rcnt[g_jl] : 1;
        if (g_jl >= 0) {
            g_bb0 = a.row_ptr[r0 + g_jl] - b0;
            g_bb1 = a.row_ptr[r0 + g_jl + 1] - b0;
        }
    }
    const bool all_cached = ncache >= nblk;


    // dst = M^-1 src for the own rows (thread = one output row of a node),
    // also into gdst unless NULL; f(element index, value) sees every result
    auto apply_minv = [&](const float *src, float *dst, float *gdst, auto &&f) {
        for (int j0 = 0; j0 < rows; j0 += ROWS_PER_PASS) {
            const int jl = j0 + grp;
            if (in_grp && jl < rows) {
                const float4 *mv = reinterpret_cast<const float4 *>(Ms + jl * 144 + rr * 12);
                const float4 *sv = reinterpret_cast<const float4 *>(src + jl * 12);
                float4 m4[3], s4[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    m4[q] = mv[q];
                    s4[q] = sv[q];
                }
                const float v = dot12(m4, s4);
                const int e = jl * 12 + rr;
                dst[e] = v;
                if (gdst) gdst[12 * r0 + e] = v;
                f(e, v);
            }
        }
    };

    // ---- set-up: r = b, d = 0, z = M^-1 r, p = z (the block columns' copies
    // were formed above); ||b|| comes with the r.r of the first iteration ----
    apply_minv(rs, zs, nullptr, [&](int, float) {});
    if (t < 6) {
        float zi = 0.f;
        for (int k = 0; k < 6; ++k) zi += Mp[6 * t + k] * s_rp[k];
        s_zp[t] = zi;
        s_pp[t] = zi;
    }
    __syncthreads();
    for (int i = t; i < rows * 12; i += NT) ps[i] = zs[i];
    const int n_items = nblk * 3;
    float res0 = 0.f;   // ||b|| (thread 0)
    if (a.n_iter == 0) {   // no iteration: ||b|| for the statistics by one reduction
        AT rr0 = A::zero();
        for (int i = t; i < rows * 12; i += NT) rr0 = A::madd(rr0, rs[i], rs[i]);
        AT vv[1] = {rr0};
        block_sum_n<DT, NT, 1>(vv, s_red);
        if (t == 0) *part_at<DT>(a.part, 0, cta) = block_sum_get<DT, NT>(s_red, 0);
        if (!ed_grid_sync(a.bar, a.status, nb + a.bar_extra, target, &s_flag, a.wait_ns)) {
            fail();
            return;
        }
        sum_partials<DT, NT, 1>(a.part, nb, s_red2);
        AT v = sum_partials_get<DT, NT, 1>(s_red2, 0);
#pragma unroll
        for (int i = 0; i < 6; ++i) v = A::madd(v, s_rp[i], s_rp[i]);
        res0 = sqrtf(A::to_float(v));
    }

    // The search direction of every block column is kept here, in step with
    // its owner: z_l <- z_l - alpha s_l, p_l <- z_l + beta p_l with the
    // owner's published s = M^-1 q, so one grid barrier per iteration
    // suffices.  The first PCG_RI float4 items of s per thread stay in
    // registers from the load after the barrier to the update.
    float4 sr[PCG_RI];
    auto stage_issue = [&](const float *sg) {
#pragma unroll
        for (int u = 0; u < PCG_RI; ++u) {
            const int i = t + u * NT;
            if (i < n_items) {
                const int lb = i / 3, q4 = i - 3 * lb;
                sr[u] = __ldcg(reinterpret_cast<const float4 *>(sg + 12 * lc[lb]) + q4);
            }
        }
    };
    auto col_update = [&](float4 &z4, float4 &p4, const float4 s4, float alpha, float beta) {
        z4 = make_float4(__fmaf_rn(-alpha, s4.x, z4.x), __fmaf_rn(-alpha, s4.y, z4.y), __fmaf_rn(-alpha, s4.z, z4.z),
                         __fmaf_rn(-alpha, s4.w, z4.w));
        p4 = make_float4(__fmaf_rn(beta, p4.x, z4.x), __fmaf_rn(beta, p4.y, z4.y), __fmaf_rn(beta, p4.z, z4.z),
                         __fmaf_rn(beta, p4.w, z4.w));
    };
    auto stage_finish = [&](const float *sg, float alpha, float beta) {
#pragma unroll
        for (int u = 0; u < PCG_RI; ++u) {
            const int i = t + u * NT;
            if (i < n_items) {
                const int lb = i / 3, q4 = i - 3 * lb;
                float4 *zp4 = reinterpret_cast<float4 *>(zb + (size_t)lb * 12) + q4;
                float4 *pp4 = reinterpret_cast<float4 *>(pb + (size_t)lb * 12) + q4;
                float4 z4 = *zp4, p4 = *pp4;
                col_update(z4, p4, sr[u], alpha, beta);
                *zp4 = z4;
                *pp4 = p4;
            }
        }
        // large CTA shares: the remaining items load s now
        for (int i = t + PCG_RI * NT; i < n_items; i += NT) {
            const int lb = i / 3, q4 = i - 3 * lb;
            const float4 s4 = __ldcg(reinterpret_cast<const float4 *>(sg + 12 * lc[lb]) + q4);
            float4 *zp4 = reinterpret_cast<float4 *>(zb + (size_t)lb * 12) + q4;
            float4 *pp4 = reinterpret_cast<float4 *>(pb + (size_t)lb * 12) + q4;
            float4 z4 = *zp4, p4 = *pp4;
            col_update(z4, p4, s4, alpha, beta);
            *zp4 = z4;
            *pp4 = p4;
        }
    };

    float rr_last = res0 * res0;   // ||r||^2 of the last residual (thread 0)
    bool breakdown = false;        // the same in every CTA: it follows from the summed p.q
    int it = 0;
    for (; it < a.n_iter; ++it) {
        float *sg = (it & 1) ? a.s1 : a.s0;                       // published s = M^-1 q (double buffer)
        double *part = a.part + (size_t)(it & 1) * ED_MAX_PCG_GRID * PCG_NC;   // partials (double buffer)
        __syncthreads();
        if (!h_ready) {   // the blocks, copied during the set-up
            if (!ed_mbar_wait(&s_mbar[1], 0, a.wait_ns)) {
                atomicCAS(a.status, ED_OK, ED_ERR_TIMEOUT);
                ed_mbar_wait(&s_mbar[1], 0);
                fail();
                return;
            }
            h_ready = true;
        }
        if (t >= NT - 6) {   // the last warp: H_pp p_pose, needed after the barrier
            const int i = t - (NT - 6);
            float h = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) h += Hpp[6 * i + k] * s_pp[k];
            s_hp[i] = h;
        }
        // ---- q = H p for the own rows (thread = one output row of one of
        // the S splits of a row's blocks), partials C p of the pose rows ----
        AT cp[6] = {A::zero(), A::zero(), A::zero(), A::zero(), A::zero(), A::zero()};
        for (int j0 = 0; j0 < rows; j0 += NG) {
            int jl = j0 + grp, sp = 0, S = 1, bb0 = g_bb0, bb1 = g_bb1;
            if (split_rows && in_grp) {   // (one pass: the group's row and block range, formed before the loop)
                jl = g_jl;
                sp = g_sp;
                S = g_S;
            } else if (in_grp && jl < rows) {
                bb0 = a.row_ptr[r0 + jl] - b0;
                bb1 = a.row_ptr[r0 + jl + 1] - b0;
            }
            if (in_grp && jl >= 0 && jl < rows) {
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
                auto madd4 = [](float acc, float4 h, float4 p) {
                    return fmaf(h.w, p.w, fmaf(h.z, p.z, fmaf(h.y, p.y, fmaf(h.x, p.x, acc))));
                };
                int lb = bb0 + sp;
                if (all_cached) {   // every block in shared memory: shared-memory loads only
                    for (; lb + S < bb1; lb += 2 * S) {
                        const float4 *ha = reinterpret_cast<const float4 *>(Hs + (size_t)lb * 144 + rr * 12);
                        const float4 *hb = reinterpret_cast<const float4 *>(Hs + (size_t)(lb + S) * 144 + rr * 12);
                        const float4 *pa = reinterpret_cast<const float4 *>(pb + (size_t)lb * 12);
                        const float4 *pbb = reinterpret_cast<const float4 *>(pb + (size_t)(lb + S) * 12);
                        const float4 ha0 = ha[0], ha1 = ha[1], ha2 = ha[2], hb0 = hb[0], hb1 = hb[1], hb2 = hb[2];
                        const float4 pa0 = pa[0], pa1 = pa[1], pa2 = pa[2], pb0 = pbb[0], pb1 = pbb[1], pb2 = pbb[2];
                        acc0 = madd4(madd4(acc0, ha0, pa0), hb0, pb0);
                        acc1 = madd4(madd4(acc1, ha1, pa1), hb1, pb1);
                        acc2 = madd4(madd4(acc2, ha2, pa2), hb2, pb2);
                    }
                    if (lb < bb1) {
                        const float4 *ha = reinterpret_cast<const float4 *>(Hs + (size_t)lb * 144 + rr * 12);
                        const float4 *pa = reinterpret_cast<const float4 *>(pb + (size_t)lb * 12);
                        acc0 = madd4(acc0, ha[0], pa[0]);
                        acc1 = madd4(acc1, ha[1], pa[1]);
                        acc2 = madd4(acc2, ha[2], pa[2]);
                    }
                    lb = bb1;
                }
                auto hrow_of = [&](int lb) {
                    return lb < ncache ? reinterpret_cast<const float4 *>(Hs + (size_t)lb * 144 + rr * 12)
                                       : reinterpret_cast<const float4 *>(a.bsr + (size_t)(b0 + lb) * 144 + rr * 12);
                };
                // two blocks per step, every load of both before the first product
                for (; lb + S < bb1; lb += 2 * S) {
                    const float4 *ha = hrow_of(lb), *hb = hrow_of(lb + S);
                    const float4 *pa = reinterpret_cast<const float4 *>(pb + (size_t)lb * 12);
                    const float4 *pbb = reinterpret_cast<const float4 *>(pb + (size_t)(lb + S) * 12);
                    const float4 ha0 = ha[0], ha1 = ha[1], ha2 = ha[2], hb0 = hb[0], hb1 = hb[1], hb2 = hb[2];
                    const float4 pa0 = pa[0], pa1 = pa[1], pa2 = pa[2], pb0 = pbb[0], pb1 = pbb[1], pb2 = pbb[2];
                    acc0 = madd4(madd4(acc0, ha0, pa0), hb0, pb0);
                    acc1 = madd4(madd4(acc1, ha1, pa1), hb1, pb1);
                    acc2 = madd4(madd4(acc2, ha2, pa2), hb2, pb2);
                }
                if (lb < bb1) {
                    const float4 *ha = hrow_of(lb);
                    const float4 *pa = reinterpret_cast<const float4 *>(pb + (size_t)lb * 12);
                    acc0 = madd4(acc0, ha[0], pa[0]);
                    acc1 = madd4(acc1, ha[1], pa[1]);
                    acc2 = madd4(acc2, ha[2], pa[2]);
                }
                qsplit[grp * 12 + rr] = acc0 + acc1 + acc2;
            }
            __syncthreads();
            // the splits of a row in a fixed order, plus the pose coupling C_j^T p_pose
            const int jr = j0 + grp;
            if (in_grp && jr < rows) {
                float qv = 0.f;
                if (split_rows) {
                    const int f = s_rfirst[jr], n = s_rcnt[jr];
                    for (int q = 0; q < n; ++q) qv += qsplit[(f + q) * 12 + rr];
                } else {
                    qv = qsplit[grp * 12 + rr];
                }
                const float *C = Cs + jr * 72;
#pragma unroll
                for (int s = 0; s < 6; ++s) qv += C[12 * s + rr] * s_pp[s];
                qs[jr * 12 + rr] = qv;
                const float pv = ps[jr * 12 + rr];
#pragma unroll
                for (int s = 0; s < 6; ++s) cp[s] = A::madd(cp[s], C[12 * s + rr], pv);
            }
            __syncthreads();   // qsplit is reused by the next pass; q complete after the last
        }
        // ---- s = M^-1 q for the own rows (published); partials of p.q, q.z,
        // q.s, r.z, r.r, r.q, q.q over the own rows ----
        {
            AT pq = A::zero(), qz = A::zero(), qq2 = A::zero(), rz = A::zero(), r2 = A::zero(), rq = A::zero(),
               q2 = A::zero();
            apply_minv(qs, ss, sg, [&](int e, float sv) {
                const float qv = qs[e], rv = rs[e], zv = zs[e];
                pq = A::madd(pq, ps[e], qv);
                qz = A::madd(qz, qv, zv);
                qq2 = A::madd(qq2, qv, sv);
                rz = A::madd(rz, rv, zv);
                r2 = A::madd(r2, rv, rv);
                rq = A::madd(rq, rv, qv);
                q2 = A::madd(q2, qv, qv);
            });
            AT vv[PCG_NC] = {pq, qz, qq2, rz, r2, rq, q2, cp[0], cp[1], cp[2], cp[3], cp[4], cp[5]};
            block_sum_bfly<DT, NT, PCG_NC>(vv, s_red);
            if (t < PCG_NC) *part_at<DT>(part, t, cta) = block_sum_get<DT, NT>(s_red, t);
        }
        if (!ed_grid_sync(a.bar, a.status, nb + a.bar_extra, target, &s_flag, a.wait_ns)) {
            fail();
            return;
        }
        stage_issue(sg);
        // ---- the sums of the partials; warp 0 adds the pose rows (q_p =
        // sum C p + H_pp p_p, s_p = M_p q_p; lane i < 6 holds entry i) and
        // their terms, takes the loop tests, forms alpha and beta and hands
        // them to the CTA ----
        // r.q and q.q serve only ||r'||^2 after the last iteration: not loaded before
        sum_partials<DT, NT, PCG_NC>(part, nb, s_red2, it + 1 < a.n_iter ? (1u << 5) | (1u << 6) : 0u);
        float qpi = 0.f, spi = 0.f;   // lanes i < 6 of warp 0: q_p[i], s_p[i]
        AT rq_t = A::zero(), q2_t = A::zero();   // thread 0: r.q and q.q
        if (t < 32) {
            const int i = t < 6 ? t : 0;
            const float qi = A::to_float(sum_partials_get<DT, NT, PCG_NC>(s_red2, 7 + i)) + s_hp[i];
            float si = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) si += Mp[6 * i + k] * __shfl_sync(0xffffffffu, qi, k);
            const float ppi = s_pp[i], zpi = s_zp[i], rpi = s_rp[i];
            AT tm[7];
            tm[0] = A::madd(A::zero(), ppi, qi);
            tm[1] = A::madd(A::zero(), qi, zpi);
            tm[2] = A::madd(A::zero(), qi, si);
            tm[3] = A::madd(A::zero(), rpi, zpi);
            tm[4] = A::madd(A::zero(), rpi, rpi);
            tm[5] = A::madd(A::zero(), rpi, qi);
            tm[6] = A::madd(A::zero(), qi, qi);
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                if (t >= 6) tm[k] = A::zero();
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) tm[k] = A::add(tm[k], A::shfl_down(tm[k], o));
            }
            qpi = qi;
            spi = si;
            if (t == 0) {
                AT tot[7];
#pragma unroll
                for (int k = 0; k < 7; ++k) tot[k] = A::add(sum_partials_get<DT, NT, PCG_NC>(s_red2, k), tm[k]);
                rq_t = tot[5];
                q2_t = tot[6];
                // r.z and r.r of the current residual: the tests of the loop head
                const float rho = A::to_float(tot[3]);
                rr_last = A::to_float(tot[4]);
                if (it == 0) res0 = sqrtf(fmaxf(rr_last, 0.f));   // r = b at the start
                int ctl = 0;
                float al = 0.f, be = 0.f;
                if (!(rho > 0.f) || (a.tol > 0.f && sqrtf(rr_last) <= a.tol * res0)) {
                    ctl = 1;
                } else {
                    const float pqt = A::to_float(tot[0]);
                    if (!(pqt > 0.f)) {
                        if (cta == 0) atomicCAS(a.status, ED_OK, ED_ERR_BREAKDOWN);
                        ctl = 2;
                    } else {
                        al = rho / pqt;
                        // r'.z' = r.z - 2 alpha q.z + alpha^2 q.s (z' = z - alpha s, M^-1 symmetric)
                        const float rho_next = rho - 2.f * al * A::to_float(tot[1]) + al * al * A::to_float(tot[2]);
                        be = rho_next / rho;
                    }
                }
                s_ab[0] = al;
                s_ab[1] = be;
                s_ctl = ctl;
            }
        }
        __syncthreads();
        {
            const int ctl = s_ctl;
            if (ctl != 0) {   // the same decision in every CTA: it follows from the summed partials
                breakdown = ctl == 2;
                break;
            }
        }
        const float alpha = s_ab[0], beta = s_ab[1];
        // ---- updates: own rows, block columns, pose (warp 0; every reader of
        // the pose parts has passed the barrier above) ----
        // (own rows from the last thread down: the first threads also take the
        // block-column items beyond the first NT)
        for (int i = NT - 1 - t; i < rows * 12; i += NT) {
            ds[i] = __fmaf_rn(alpha, ps[i], ds[i]);
            rs[i] = __fmaf_rn(-alpha, qs[i], rs[i]);
            const float zn = __fmaf_rn(-alpha, ss[i], zs[i]);
            zs[i] = zn;
            ps[i] = __fmaf_rn(beta, ps[i], zn);
        }
        stage_finish(sg, alpha, beta);
        if (t < 6) {
            s_dp[t] = __fmaf_rn(alpha, s_pp[t], s_dp[t]);
            s_rp[t] = __fmaf_rn(-alpha, qpi, s_rp[t]);
            const float zn = __fmaf_rn(-alpha, spi, s_zp[t]);
            s_zp[t] = zn;
            s_pp[t] = __fmaf_rn(beta, s_pp[t], zn);
        }
        // ||r'||^2 = r.r - 2 alpha r.q + alpha^2 q.q (reported after the last iteration)
        if (t == 0) rr_last = rr_last - 2.f * alpha * A::to_float(rq_t) + alpha * alpha * A::to_float(q2_t);
    }
    __syncthreads();
    // solution of the CTA's rows (and of the pose: CTA 0), and the update
    // x += d, pose += d_pose unless the solve broke down.  No wait follows the
    // last barrier, so in normal operation either every CTA gets here or none
    // does; an error reported meanwhile (a wait elsewhere that ran out) also
    // withholds the update.
    if (t == 0) s_flag = *(volatile int *)a.status == ED_OK;
    __syncthreads();
    if (!s_flag) breakdown = true;
    for (int i = t; i < rows * 12; i += NT) {
        const size_t gi = 12 * (size_t)r0 + i;
        const float dv = ds[i];
        a.d[gi] = dv;
        if (!breakdown) {
            if (a.xm) {
                const double v = a.xm[gi] + (double)dv;
                a.xm[gi] = v;
                a.x[gi] = (float)v;
            } else {
                a.x[gi] += dv;
            }
        }
    }
    if (cta == 0 && t < 6) {
        a.d[P + t] = s_dp[t];
        if (!breakdown) a.pose[t] += (double)s_dp[t];
    }
    if (cta == 0 && t == 0 && a.stats) {
        a.stats->pcg_iters = it;
        a.stats->pcg_res0 = (double)res0;
        a.stats->pcg_res = sqrt((double)fmaxf(rr_last, 0.f));
        a.stats->status = *(volatile int *)a.status;
    }
}

template <typename DT, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_pcg(PcgArgs a)
{
    // (no early trigger: the next point pass reads x and the pose through the
    // read-only path, so it must not be alive while this kernel writes them)
    if (!a.load_before_wait) ed_pdl_wait();
    pcg_body<DT, NT>(a, blockIdx.x, gridDim.x);
}

// many independent problems in one persistent launch: CTAs [cta_first[p],
// cta_first[p+1]) solve problem p with their own barrier and partials
struct PcgBatchParams {
    int count;
    int cta_first[ED_MAX_BATCH_LAUNCH + 1];
    PcgArgs probs[ED_MAX_BATCH_LAUNCH];
};

template <typename DT, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_pcg_batch(const __grid_constant__ PcgBatchParams b)
{
    int p = 0;
    while (p + 1 < b.count && (int)blockIdx.x >= b.cta_first[p + 1]) ++p;
    pcg_body<DT, NT>(b.probs[p], (int)blockIdx.x - b.cta_first[p], (unsigned)(b.cta_first[p + 1] - b.cta_first[p]));
}

// the dynamic shared-memory limit of every PCG kernel, raised once per device
static std::mutex g_attr_mutex;
static bool g_attr_done[256];

static ed_status pcg_set_attributes()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return ED_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (g_attr_done[dev]) return ED_OK;
    const int big = PCG_SMEM_MAX, small = PCG_SMEM_MAX_256;
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg<float, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg<double, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, small));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg<double, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, small));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch<float, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch<double, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, small));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch<double, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, small));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg<PcgFp64, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg<PcgFp64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, small));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch<PcgFp64, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    ED_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch<PcgFp64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, small));
    g_attr_done[dev] = true;
    return ED_OK;
}

// balanced row partition of one problem over `grid` CTAs (by block count, at
// least one row each) and its shared-memory plan for NT threads per CTA
ed_status ed_pcg_make_plan(const int *row_ptr_host, int m, int grid, int nt, ed_pcg_plan_t *pl, int *rows_start)
{
    if (grid < 1 || grid > m || grid > ED_MAX_PCG_GRID || (nt != 256 && nt != 512)) return ED_ERR_ARG;
    const int nnzb = row_ptr_host[m];
    int r = 0;
    rows_start[0] = 0;
    for (int c = 1; c < grid; ++c) {
        const long want = (long)nnzb * c / grid;
        while (r < m && row_ptr_host[r] < want) ++r;
        if (r < rows_start[c - 1] + 1) r = rows_start[c - 1] + 1;
        if (r > m - (grid - c)) r = m - (grid - c);
        rows_start[c] = r;
    }
    rows_start[grid] = m;
    int max_rows = 0, max_blk = 0;
    for (int c = 0; c < grid; ++c) {
        const int rw = rows_start[c + 1] - rows_start[c];
        const int nbk = row_ptr_host[rows_start[c + 1]] - row_ptr_host[rows_start[c]];
        if (rw > max_rows) max_rows = rw;
        if (nbk > max_blk) max_blk = nbk;
    }
    const size_t smem_max = nt == 512 ? PCG_SMEM_MAX : PCG_SMEM_MAX_256;
    const PcgSmem base = pcg_smem_layout(max_rows, max_blk, 0, nt);
    const size_t base_bytes = base.total * sizeof(float);
    if (base_bytes > smem_max) return ED_ERR_CAPACITY;
    int ncache = (int)((smem_max - base_bytes) / (144 * sizeof(float)));
    if (ncache > max_blk) ncache = max_blk;
    pl->grid = grid;
    pl->nt = nt;
    pl->ncache = ncache;
    pl->max_rows = max_rows;
    pl->max_blk = max_blk;
    pl->smem = pcg_smem_layout(max_rows, max_blk, ncache, nt).total * sizeof(float);
    return ED_OK;
}

// plan of the single-problem solve (one 512-thread CTA per SM); called at graph
// build with the row pointer copied to the host
ed_status ed_pcg_plan(ed_context *ctx, const int *row_ptr_host, cudaStream_t st)
{
    ed_status s = pcg_set_attributes();
    if (s != ED_OK) return s;
    const int m = ctx->m;
    int grid = ctx->num_sms;
    if (grid > ED_MAX_PCG_GRID) grid = ED_MAX_PCG_GRID;
    if (grid > m) grid = m;
    int *rows_start = ctx->pinned;   // pinned: the copy below needs no synchronisation
    ed_pcg_plan_t pl;
    if ((s = ed_pcg_make_plan(row_ptr_host, m, grid, 512, &pl, rows_start)) != ED_OK) return s;
    ctx->pcg = pl;
    if (row_ptr_host != ctx->row_ptr_host) memcpy(ctx->row_ptr_host, row_ptr_host, sizeof(int) * (m + 1));
    ED_CUDA_TRY(cudaMemcpyAsync(ctx->pcg_rows, rows_start, sizeof(int) * (grid + 1), cudaMemcpyHostToDevice, st));
    return ED_OK;
}

static ed_status pcg_fill_args(ed_context *ctx, const ed_pcg_plan_t &pl, const int *cta_rows,
                               const ed_solver_params *prm, float *x, double *xm, double *pose, ed_stats *stats,
                               PcgArgs &a)
{
    if (!x || !pose || ((uintptr_t)x & 15)) return ED_ERR_ARG;
    a.x = x;
    a.xm = ed_is_mixed(prm->precision) ? xm : nullptr;
    a.pose = pose;
    const size_t P = ctx->vec_stride;
    a.m = ctx->m;
    a.n_iter = prm->n_pcg;
    a.tol = prm->pcg_tol;
    a.row_ptr = ctx->row_ptr;
    a.col = ctx->col;
    a.cta_rows = cta_rows;
    a.n_cache = pl.ncache;
    a.max_rows = pl.max_rows;
    a.max_blk = pl.max_blk;
    a.bsr = ctx->bsr;
    a.pnode = ctx->pnode;
    a.minv = ctx->minv;
    a.pose_blk = ctx->pose_blk;
    a.grad = ctx->grad;
    a.d = ctx->vec;
    a.s0 = ctx->vec + 3 * P;
    a.s1 = ctx->vec + 4 * P;
    a.part = ctx->pcg_part;
    a.bar = (unsigned *)(ctx->misc + MI_BAR);
    a.bar_extra = (unsigned)ctx->bar_extra;
    a.wait_ns = ctx->wait_ns;
    a.status = ctx->misc + MI_STATUS;
    a.stats = stats;
    a.load_before_wait = 0;
    // every vector is read as float4 rows: 16-byte alignment is required
    const float *vv[3] = {a.d, a.s0, a.s1};
    for (int i = 0; i < 3; ++i)
        if ((uintptr_t)vv[i] & 15) return ED_ERR_STATE;
    if (((uintptr_t)a.bsr & 15) || ((uintptr_t)a.minv & 15)) return ED_ERR_STATE;
    return ED_OK;
}


ed_status ed_pcg_solve(ed_context *ctx, const ed_solver_params *prm, float *x, double *xm, double *pose,
                       ed_stats *stats, cudaStream_t st)
{
    if (ctx->pcg.grid <= 0) return ED_ERR_STATE;
    PcgArgs a;
    ed_status s = pcg_fill_args(ctx, ctx->pcg, ctx->pcg_rows, prm, x, xm, pose, stats, a);
    if (s != ED_OK) return s;
    // the stream predecessor is k_fin_totals unless the Levenberg-Marquardt
    // stage comes between (its kernels are launched without triggers)
    a.load_before_wait = prm->lm_accept ? 0 : 1;
    // (the arrival count was cleared by k_fin_totals, after the finalisation)
    void *args[] = {&a};
    ed_tm_begin(ctx, ED_KERNEL_PCG, st);
    ed_note_launch();
    const void *fn = prm->precision == ED_PRECISION_MIXED        ? (const void *)k_pcg<double, 512>
                     : prm->precision == ED_PRECISION_MIXED_FP64 ? (const void *)k_pcg<PcgFp64, 512>
                                                                 : (const void *)k_pcg<float, 512>;
    cudaError_t e = ed_launch_coop(fn, ctx->pcg.grid, 512, args, ctx->pcg.smem, st, true);
    ed_tm_end(ctx, ED_KERNEL_PCG, st);
    if (e != cudaSuccess) {
        fprintf(stderr, "libed: PCG launch failed: %s\n", cudaGetErrorString(e));
        return ED_ERR_CUDA;
    }
    return ED_OK;
}

// Plan of one batched launch: CTAs split over the problems in proportion to
// their stored blocks (at least one each, at most one per node row), each
// problem's rows partitioned over its CTAs; row starts go to pcg_rows_b.
ed_status ed_pcg_batch_plan(ed_context *const *ctxs, int count, int nt, int grid_total, ed_pcg_batch_plan_t *bp)
{
    ed_status s = pcg_set_attributes();
    if (s != ED_OK) return s;
    if (count < 1 || count > ED_MAX_BATCH_LAUNCH || (nt != 256 && nt != 512)) return ED_ERR_ARG;
    if (grid_total < count) return ED_ERR_CAPACITY;
    long tot = 0;
    for (int p = 0; p < count; ++p) tot += ctxs[p]->nnzb;
    int alloc[ED_MAX_BATCH_LAUNCH];
    int used = 0;
    for (int p = 0; p < count; ++p) {
        long c = tot > 0 ? (long)grid_total * ctxs[p]->nnzb / tot : 1;
        if (c < 1) c = 1;
        if (c > ctxs[p]->m) c = ctxs[p]->m;
        if (c > ED_MAX_PCG_GRID) c = ED_MAX_PCG_GRID;
        alloc[p] = (int)c;
        used += (int)c;
    }
    // trim or hand out the remainder, largest work per CTA first
    while (used > grid_total) {
        int best = -1;
        for (int p = 0; p < count; ++p)
            if (alloc[p] > 1 && (best < 0 || (double)ctxs[p]->nnzb / alloc[p] < (double)ctxs[best]->nnzb / alloc[best]))
                best = p;
        if (best < 0) return ED_ERR_CAPACITY;
        --alloc[best];
        --used;
    }
    while (used < grid_total) {
        int best = -1;
        for (int p = 0; p < count; ++p)
            if (alloc[p] < ctxs[p]->m && alloc[p] < ED_MAX_PCG_GRID &&
                (best < 0 || (double)ctxs[p]->nnzb / alloc[p] > (double)ctxs[best]->nnzb / alloc[best]))
                best = p;
        if (best < 0) break;
        ++alloc[best];
        ++used;
    }
    bp->count = count;
    bp->nt = nt;
    bp->smem = 0;
    bp->cta_first[0] = 0;
    static thread_local int rows_start[ED_MAX_PCG_GRID + 1];
    for (int p = 0; p < count; ++p) {
        ed_context *c = ctxs[p];
        if (!c->have_graph || c->build_pending) return ED_ERR_STATE;   // (the batch read the counts at creation)
        if ((s = ed_pcg_make_plan(c->row_ptr_host, c->m, alloc[p], nt, &bp->plan[p], rows_start)) != ED_OK) return s;
        ED_CUDA_TRY(cudaMemcpy(c->pcg_rows_b, rows_start, sizeof(int) * (alloc[p] + 1), cudaMemcpyHostToDevice));
        bp->cta_first[p + 1] = bp->cta_first[p] + alloc[p];
        if (bp->plan[p].smem > bp->smem) bp->smem = bp->plan[p].smem;
    }
    bp->grid = bp->cta_first[count];
    return ED_OK;
}

// one persistent launch for the PCG solves of a planned group of problems
ed_status ed_pcg_solve_batch(ed_context *const *ctxs, const ed_pcg_batch_plan_t *bp, const ed_solver_params *const *prm,
                             float *const *x, double *const *xm, double *const *pose, ed_stats *const *stats,
                             cudaStream_t st)
{
    const int count = bp->count;
    const int prec = prm[0]->precision;
    PcgBatchParams b;
    memset(&b, 0, sizeof(b));
    b.count = count;
    for (int p = 0; p <= count; ++p) b.cta_first[p] = bp->cta_first[p];
    for (int p = 0; p < count; ++p) {
        if (prm[p]->precision != prec) return ED_ERR_ARG;
        ed_status s = pcg_fill_args(ctxs[p], bp->plan[p], ctxs[p]->pcg_rows_b, prm[p], x[p], xm[p], pose[p], stats[p],
                                    b.probs[p]);
        if (s != ED_OK) return s;
        ED_CUDA_TRY(cudaMemsetAsync(ctxs[p]->misc + MI_BAR, 0, 2 * sizeof(int), st));
    }
    void *args[] = {&b};
    const void *fn;
    if (bp->nt == 512)
        fn = prec == ED_PRECISION_MIXED        ? (const void *)k_pcg_batch<double, 512>
             : prec == ED_PRECISION_MIXED_FP64 ? (const void *)k_pcg_batch<PcgFp64, 512>
                                               : (const void *)k_pcg_batch<float, 512>;
    else
        fn = prec == ED_PRECISION_MIXED        ? (const void *)k_pcg_batch<double, 256>
             : prec == ED_PRECISION_MIXED_FP64 ? (const void *)k_pcg_batch<PcgFp64, 256>
                                               : (const void *)k_pcg_batch<float, 256>;
    ed_note_launch();
    // (a timing hook set on the group's first context brackets the launch)
    ed_tm_begin(ctxs[0], ED_KERNEL_PCG, st);
    cudaError_t e = ed_launch_coop(fn, bp->grid, bp->nt, args, bp->smem, st, false);
    if (e == cudaSuccess) ed_tm_end(ctxs[0], ED_KERNEL_PCG, st);
    if (e != cudaSuccess) {
        fprintf(stderr, "libed: batched PCG launch failed: %s\n", cudaGetErrorString(e));
        return ED_ERR_CUDA;
    }
    return ED_OK;
}
