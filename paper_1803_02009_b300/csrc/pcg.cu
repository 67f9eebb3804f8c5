// pcg.cu -- block-Jacobi preconditioned conjugate gradients on the normal
// equations of one Gauss-Newton step (Sec. II.F), as one persistent
// cooperative kernel.
//
// H is a symmetric block-sparse matrix over the m nodes (12x12 blocks, both
// triangles stored, row-major blocks) bordered by the 6 pose unknowns:
// pose-node blocks C_j (6x12) and a 6x6 pose block.  Each CTA (one per SM)
// owns a contiguous range of node rows, balanced by block count at graph
// build; CTA 0 also owns the pose rows.  For the whole solve a CTA keeps in
// shared memory its rows' blocks (as many as fit; the rest stream from L2),
// block inverses, pose-node blocks and its slices of d, r, z, p, q.  Per PCG
// iteration it forms the search direction of every block column it touches,
// p_l = z_l + beta p_l(prev), from the owners' z and previous p (double
// buffer), which it loads in the same round of loads as the reduction that
// follows the second barrier; multiplies from shared memory (several thread
// groups per row when a CTA has few rows) and meets the other CTAs at two
// bounded grid barriers (after q = H p for p.q and the pose row, after
// z = M^-1 r for r.z).  Reductions are per-CTA partials summed in a fixed
// order by every CTA: deterministic.
#include <mutex>

#include "ed_internal.cuh"

#define PCG_SMEM_MAX (200 * 1024)      // one 512-thread CTA per SM
#define PCG_SMEM_MAX_256 (100 * 1024)  // two 256-thread CTAs per SM

#define PCG_RI 2                       // staged column items per thread held in registers

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
    float *d, *z, *p0, *p1;  // global vectors (z and p are read by other CTAs)
    double *part;            // [2][ED_PCG_PART][ED_MAX_PCG_GRID], component-major
    unsigned *bar;           // arrival count
    int *status;
    ed_stats *stats;
};

// Accumulation of the PCG dot products and norms.  FP32 mode: float.  Mixed
// mode: float-float (hi + lo, about 44 significant bits) on the FP32 pipe --
// each product is formed exactly (a b = p + e with e = fma(a, b, -p)) and
// summed by error-free two-sums; on B300 the FP64 rate is a small fraction of
// the FP32 rate, so the extended precision is kept off the FP64 units.  The
// per-CTA partials between CTAs are stored as double.
template <typename DT> struct PcgAcc;

template <> struct PcgAcc<float> {
    typedef float T;
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ T madd(T acc, float a, float b) { return acc + a * b; }
    static __device__ __forceinline__ T add(T x, T y) { return x + y; }
    static __device__ __forceinline__ T shfl(T x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
    static __device__ __forceinline__ T from_double(double d) { return (float)d; }
    static __device__ __forceinline__ double to_double(T x) { return (double)x; }
    static __device__ __forceinline__ float to_float(T x) { return x; }
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
    static __device__ __forceinline__ T from_double(double d)
    {
        const float hi = (float)d;
        return make_float2(hi, (float)(d - (double)hi));
    }
    static __device__ __forceinline__ double to_double(T x) { return (double)x.x + (double)x.y; }
    static __device__ __forceinline__ float to_float(T x) { return x.x + x.y; }
};

// component w of the partials of CTA c
__device__ __forceinline__ double *part_at(double *part, int w, int c) { return part + (size_t)w * ED_MAX_PCG_GRID + c; }

// sums the NC components of all CTA partials: NT / NCP threads per
// component stride over the CTAs (one round of loads for up to 4x that many
// CTAs), then a fixed shuffle tree and a fixed-order sum of the warp results
// that every thread forms itself (one CTA barrier), so every CTA and every
// thread gets the same values.  `sh` must not be in use by other code
// between two calls.
template <typename DT, int NT, int NC>
__device__ __forceinline__ void sum_partials(const double *part, int nb, typename PcgAcc<DT>::T (*sh)[8],
                                             typename PcgAcc<DT>::T (&out)[NC])
{
    typedef PcgAcc<DT> A;
    constexpr int NCP = NC <= 1 ? 1 : NC <= 2 ? 2 : NC <= 4 ? 4 : 8;
    constexpr int TPC = NT / NCP;       // threads per component
    constexpr int WPC = TPC / 32;       // warps per component
    const int lane = threadIdx.x & 31, w = threadIdx.x / TPC, sub = threadIdx.x % TPC;
    typename A::T s = A::zero();
    if (w < NC) {
        const double *src = part + (size_t)w * ED_MAX_PCG_GRID;
#pragma unroll 4
        for (int c = sub; c < nb; c += TPC) s = A::add(s, A::from_double(__ldcg(src + c)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl(s, o));
    if (lane == 0) sh[threadIdx.x >> 5][0] = s;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        typename A::T r = A::zero();
#pragma unroll
        for (int k = 0; k < WPC; ++k) r = A::add(r, sh[c * WPC + k][0]);
        out[c] = r;
    }
}

// block reduction of NV values per thread: after one CTA barrier,
// block_sum_get(c) gives component c (fixed order) to any thread that asks
template <typename DT, int NT, int NV>
__device__ __forceinline__ void block_sum_n(typename PcgAcc<DT>::T (&v)[NV], typename PcgAcc<DT>::T (*sh)[8])
{
    typedef PcgAcc<DT> A;
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

template <typename DT, int NT>
__device__ __forceinline__ typename PcgAcc<DT>::T block_sum_get(const typename PcgAcc<DT>::T (*sh)[8], int c)
{
    typedef PcgAcc<DT> A;
    typename A::T s = A::zero();
    for (int w = 0; w < NT / 32; ++w) s = A::add(s, sh[w][c]);
    return s;
}

// shared-memory carve of one CTA (in floats; every region a multiple of 4)
struct PcgSmem {
    size_t o_H, o_pb, o_po, o_lc, o_M, o_C, o_r, o_d, o_z, o_p, o_q, o_qs, total;
};

__host__ __device__ inline PcgSmem pcg_smem_layout(int rows, int nblk, int ncache, int nt)
{
    PcgSmem L;
    size_t o = 0;
    L.o_H = o; o += (size_t)ncache * 144;
    L.o_pb = o; o += (size_t)nblk * 12;            // z of the block columns, then p
    L.o_po = o; o += (size_t)nblk * 12;            // previous p of the block columns
    L.o_lc = o; o += ((size_t)nblk + 3) / 4 * 4;   // block column indices (int)
    L.o_M = o; o += (size_t)rows * 144;
    L.o_C = o; o += (size_t)rows * 72;
    L.o_r = o; o += (size_t)rows * 12;
    L.o_d = o; o += (size_t)rows * 12;
    L.o_z = o; o += (size_t)rows * 12;
    L.o_p = o; o += (size_t)rows * 12;
    L.o_q = o; o += (size_t)rows * 12;
    L.o_qs = o; o += (size_t)(nt / 12) * 12;       // split partial products of q
    L.total = o;
    return L;
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
    __shared__ AT s_red[NT / 32][8];    // block reductions
    __shared__ AT s_red2[NT / 32][8];   // sums of the CTA partials
    __shared__ float s_pp[6], s_zp[6], s_rpose[6], s_dpose[6];
    __shared__ float s_Hpp[36], s_Mp[36];

    unsigned target = 0;
    const int m = a.m;
    const int r0 = a.cta_rows[cta], r1 = a.cta_rows[cta + 1];
    const int rows = r1 - r0;
    const int b0 = a.row_ptr[r0], nblk = a.row_ptr[r1] - b0;
    const int ncache = min(nblk, a.n_cache);
    const PcgSmem L = pcg_smem_layout(a.max_rows, a.max_blk, a.n_cache, NT);
    float *Hs = sm + L.o_H, *pb = sm + L.o_pb, *po = sm + L.o_po, *Ms = sm + L.o_M, *Cs = sm + L.o_C;
    float *rs = sm + L.o_r, *ds = sm + L.o_d, *zs = sm + L.o_z, *ps = sm + L.o_p, *qs = sm + L.o_q;
    float *qsplit = sm + L.o_qs;
    int *lc = reinterpret_cast<int *>(sm + L.o_lc);
    const int t = threadIdx.x;
    const int grp = t / 12, rr = t % 12;
    const bool in_grp = grp < ROWS_PER_PASS;
    // q = H p: with few rows, S groups of 12 threads share the blocks of a row
    const int S = rows <= ROWS_PER_PASS ? ROWS_PER_PASS / rows : 1;
    const int rpp = ROWS_PER_PASS / S;   // rows per pass
    const int P = 12 * m;
    const float *Hpp = s_Hpp, *Mp = s_Mp;
    double *part0 = a.part, *part1 = a.part + (size_t)ED_MAX_PCG_GRID * ED_PCG_PART;

    if (*(volatile int *)a.status != ED_OK) return;

    // ---- the CTA's share of H, M^-1 and C into shared memory by bulk
    // asynchronous copies (inverses and pose-node blocks on mbarrier 0, needed
    // first; blocks on mbarrier 1, needed by the first q = H p); block columns
    // and b by plain loads meanwhile ----
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
    if (!ed_mbar_wait(&s_mbar[0], 0)) {
        atomicCAS(a.status, ED_OK, ED_ERR_TIMEOUT);
        ed_mbar_wait(&s_mbar[0], 0);
        ed_mbar_wait(&s_mbar[1], 0);
        return;
    }
    __syncthreads();
    bool h_ready = false;

    // z_j = Minv_j r_j for the own rows (thread = one output row); partials r.z, r.r
    auto precond = [&](AT &rz, AT &rrs) {
        for (int j0 = 0; j0 < rows; j0 += ROWS_PER_PASS) {
            const int jl = j0 + grp;
            if (in_grp && jl < rows) {
                const float4 *mv = reinterpret_cast<const float4 *>(Ms + jl * 144 + rr * 12);
                const float4 *rv = reinterpret_cast<const float4 *>(rs + jl * 12);
                float zz = 0.f;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float4 m4 = mv[q], r4 = rv[q];
                    zz += m4.x * r4.x + m4.y * r4.y + m4.z * r4.z + m4.w * r4.w;
                }
                const float rv1 = rs[jl * 12 + rr];
                zs[jl * 12 + rr] = zz;
                a.z[12 * (r0 + jl) + rr] = zz;
                rz = A::madd(rz, rv1, zz);
                rrs = A::madd(rrs, rv1, rv1);
            }
        }
    };

    // pose rows (CTA 0, thread 0): z_p = Mp r_p; adds the pose terms of r.z and r.r
    auto pose_precond = [&](AT &v1, AT &v2) {
        for (int i = 0; i < 6; ++i) {
            float zi = 0.f;
            for (int k = 0; k < 6; ++k) zi += Mp[6 * i + k] * s_rpose[k];
            a.z[P + i] = zi;
            v1 = A::madd(v1, s_rpose[i], zi);
            v2 = A::madd(v2, s_rpose[i], s_rpose[i]);
        }
    };

    // The block columns' z and previous p from their owners, loaded in the same
    // round as the reduction that follows each barrier: the first PCG_RI
    // float4 items of every thread stay in registers until beta is known, the
    // rest (large CTA shares) go through shared memory.
    float4 zr[PCG_RI], pr[PCG_RI];
    const int n_items = nblk * 3;
    auto stage_issue = [&](const float *pprev) {
#pragma unroll
        for (int u = 0; u < PCG_RI; ++u) {
            const int i = t + u * NT;
            if (i < n_items) {
                const int lb = i / 3, q4 = i - 3 * lb;
                const int l = lc[lb];
                zr[u] = __ldcg(reinterpret_cast<const float4 *>(a.z + 12 * l) + q4);
                pr[u] = pprev ? __ldcg(reinterpret_cast<const float4 *>(pprev + 12 * l) + q4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        for (int i = t + PCG_RI * NT; i < n_items; i += NT) {
            const int lb = i / 3, q4 = i - 3 * lb;
            const int l = lc[lb];
            reinterpret_cast<float4 *>(pb + (size_t)lb * 12)[q4] =
                __ldcg(reinterpret_cast<const float4 *>(a.z + 12 * l) + q4);
            if (pprev)
                reinterpret_cast<float4 *>(po + (size_t)lb * 12)[q4] =
                    __ldcg(reinterpret_cast<const float4 *>(pprev + 12 * l) + q4);
        }
        if (t < 6) s_zp[t] = __ldcg(a.z + P + t);
    };
    // p_l = z_l + beta p_l(prev) for every staged item (beta unused at the first iteration)
    auto stage_finish = [&](float beta, bool first) {
#pragma unroll
        for (int u = 0; u < PCG_RI; ++u) {
            const int i = t + u * NT;
            if (i < n_items) {
                const int lb = i / 3, q4 = i - 3 * lb;
                const float4 z4 = zr[u], p4 = pr[u];
                reinterpret_cast<float4 *>(pb + (size_t)lb * 12)[q4] =
                    first ? z4
                          : make_float4(__fmaf_rn(beta, p4.x, z4.x), __fmaf_rn(beta, p4.y, z4.y),
                                        __fmaf_rn(beta, p4.z, z4.z), __fmaf_rn(beta, p4.w, z4.w));
            }
        }
        if (!first) {
            for (int i = t + PCG_RI * NT; i < n_items; i += NT) {
                const int lb = i / 3, q4 = i - 3 * lb;
                float4 *b4 = reinterpret_cast<float4 *>(pb + (size_t)lb * 12) + q4;
                const float4 z4 = *b4, p4 = reinterpret_cast<const float4 *>(po + (size_t)lb * 12)[q4];
                *b4 = make_float4(__fmaf_rn(beta, p4.x, z4.x), __fmaf_rn(beta, p4.y, z4.y), __fmaf_rn(beta, p4.z, z4.z),
                                  __fmaf_rn(beta, p4.w, z4.w));
            }
        }
    };

    // ---- set-up: r = b, d = 0, z = M^-1 r ----
    {
        AT rz = A::zero(), rrs = A::zero();
        precond(rz, rrs);
        AT vv[2] = {rz, rrs};
        block_sum_n<DT, NT, 2>(vv, s_red);
    }
    if (t == 0) {
        AT v1 = block_sum_get<DT, NT>(s_red, 0), v2 = block_sum_get<DT, NT>(s_red, 1);
        if (cta == 0) {
            for (int i = 0; i < 6; ++i) {
                s_rpose[i] = -a.grad[P + i];
                s_dpose[i] = 0.f;
            }
            pose_precond(v1, v2);
        }
        *part_at(part0, 0, cta) = A::to_double(v1);
        *part_at(part0, 1, cta) = A::to_double(v2);
    }
    if (!ed_grid_sync(a.bar, a.status, nb, target, &s_flag)) return;
    stage_issue(nullptr);
    // the scalars of the iteration live in every thread's registers (identical values)
    AT rho, rr2s;
    float res0, beta = 0.f;
    {
        AT sums[2];
        sum_partials<DT, NT, 2>(part0, nb, s_red2, sums);
        rho = sums[0];
        rr2s = sums[1];
        res0 = sqrtf(A::to_float(sums[1]));
    }
    float qp[6];   // the pose rows of q = H p (CTA 0 thread 0 uses them for the pose update)

    int it = 0;
    for (; it < a.n_iter; ++it) {
        if (!(A::to_float(rho) > 0.f)) break;
        if (a.tol > 0.f && sqrtf(A::to_float(rr2s)) <= a.tol * res0) break;
        float *pnew = (it & 1) ? a.p1 : a.p0;
        // ---- p = z + beta p(prev): block columns (staged), own rows (published), pose ----
        stage_finish(beta, it == 0);
        for (int i = t; i < rows * 12; i += NT) {
            const float pv = it > 0 ? __fmaf_rn(beta, ps[i], zs[i]) : zs[i];
            ps[i] = pv;
            pnew[12 * r0 + i] = pv;
        }
        if (t < 6) s_pp[t] = it > 0 ? __fmaf_rn(beta, s_pp[t], s_zp[t]) : s_zp[t];
        __syncthreads();
        if (!h_ready) {   // the blocks, copied during the set-up
            if (!ed_mbar_wait(&s_mbar[1], 0)) {
                atomicCAS(a.status, ED_OK, ED_ERR_TIMEOUT);
                ed_mbar_wait(&s_mbar[1], 0);
                return;
            }
            h_ready = true;
        }
        // ---- phase A: q = H p for the own rows (thread = one output row of one
        // of the S splits of a row's blocks), partials p.q and C p ----
        AT pq = A::zero();
        AT cp[6] = {A::zero(), A::zero(), A::zero(), A::zero(), A::zero(), A::zero()};
        for (int j0 = 0; j0 < rows; j0 += rpp) {
            const int jl = j0 + grp / S, sp = grp - (grp / S) * S;
            if (in_grp && grp < rpp * S && jl < rows) {
                const int j = r0 + jl;
                const int bb0 = a.row_ptr[j] - b0, bb1 = a.row_ptr[j + 1] - b0;
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
                for (int lb = bb0 + sp; lb < bb1; lb += S) {
                    const float4 *hrow = lb < ncache ? reinterpret_cast<const float4 *>(Hs + (size_t)lb * 144 + rr * 12)
                                                     : reinterpret_cast<const float4 *>(a.bsr + (size_t)(b0 + lb) * 144 + rr * 12);
                    const float4 *pl = reinterpret_cast<const float4 *>(pb + (size_t)lb * 12);
                    const float4 h0 = hrow[0], h1 = hrow[1], h2 = hrow[2];
                    const float4 p0 = pl[0], p1 = pl[1], p2 = pl[2];
                    acc0 += h0.x * p0.x + h0.y * p0.y + h0.z * p0.z + h0.w * p0.w;
                    acc1 += h1.x * p1.x + h1.y * p1.y + h1.z * p1.z + h1.w * p1.w;
                    acc2 += h2.x * p2.x + h2.y * p2.y + h2.z * p2.z + h2.w * p2.w;
                }
                qsplit[grp * 12 + rr] = acc0 + acc1 + acc2;
            }
            __syncthreads();
            // the S splits of a row in a fixed order, plus the pose coupling C_j^T p_pose
            const int jr = j0 + grp;
            if (in_grp && grp < rpp && jr < rows) {
                float qv = 0.f;
                for (int q = 0; q < S; ++q) qv += qsplit[(grp * S + q) * 12 + rr];
                const float *C = Cs + jr * 72;
#pragma unroll
                for (int s = 0; s < 6; ++s) qv += C[12 * s + rr] * s_pp[s];
                qs[jr * 12 + rr] = qv;
                const float pv = ps[jr * 12 + rr];
                pq = A::madd(pq, pv, qv);
#pragma unroll
                for (int s = 0; s < 6; ++s) cp[s] = A::madd(cp[s], C[12 * s + rr], pv);
            }
            if (j0 + rpp < rows) __syncthreads();   // qsplit is reused by the next pass
        }
        {
            AT vv[7] = {pq, cp[0], cp[1], cp[2], cp[3], cp[4], cp[5]};
            block_sum_n<DT, NT, 7>(vv, s_red);
            if (t < 7) *part_at(part1, t, cta) = A::to_double(block_sum_get<DT, NT>(s_red, t));
        }
        if (!ed_grid_sync(a.bar, a.status, nb, target, &s_flag)) return;
        // ---- phase B: alpha (every thread), d += alpha p, r -= alpha q, z = M^-1 r ----
        float alpha;
        {
            AT sums[7];
            sum_partials<DT, NT, 7>(part1, nb, s_red2, sums);
            AT pqt = sums[0];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                float qi = A::to_float(sums[1 + i]);
#pragma unroll
                for (int k = 0; k < 6; ++k) qi += Hpp[6 * i + k] * s_pp[k];
                qp[i] = qi;
                pqt = A::madd(pqt, s_pp[i], qi);
            }
            const float pqt_f = A::to_float(pqt);
            if (!(pqt_f > 0.f)) {
                if (cta == 0 && t == 0) atomicCAS(a.status, ED_OK, ED_ERR_BREAKDOWN);
                break;
            }
            alpha = A::to_float(rho) / pqt_f;
        }
        for (int i = t; i < rows * 12; i += NT) {
            ds[i] = __fmaf_rn(alpha, ps[i], ds[i]);
            rs[i] = __fmaf_rn(-alpha, qs[i], rs[i]);
        }
        __syncthreads();
        {
            AT rz2 = A::zero(), rr2 = A::zero();
            precond(rz2, rr2);
            AT vv[2] = {rz2, rr2};
            block_sum_n<DT, NT, 2>(vv, s_red);
        }
        if (t == 0) {
            AT w1 = block_sum_get<DT, NT>(s_red, 0), w2 = block_sum_get<DT, NT>(s_red, 1);
            if (cta == 0) {
                for (int i = 0; i < 6; ++i) {
                    s_dpose[i] = __fmaf_rn(alpha, s_pp[i], s_dpose[i]);
                    s_rpose[i] = __fmaf_rn(-alpha, qp[i], s_rpose[i]);
                }
                pose_precond(w1, w2);
            }
            *part_at(part0, 0, cta) = A::to_double(w1);
            *part_at(part0, 1, cta) = A::to_double(w2);
        }
        if (!ed_grid_sync(a.bar, a.status, nb, target, &s_flag)) return;
        stage_issue(pnew);
        {
            AT sums[2];
            sum_partials<DT, NT, 2>(part0, nb, s_red2, sums);
            beta = A::to_float(sums[0]) / A::to_float(rho);
            rho = sums[0];
            rr2s = sums[1];
        }
    }
    // solution of the CTA's rows (and of the pose: CTA 0)
    for (int i = t; i < rows * 12; i += NT) a.d[12 * r0 + i] = ds[i];
    if (cta == 0 && t < 6) a.d[P + t] = s_dpose[t];
    if (cta == 0 && t == 0 && a.stats) {
        a.stats->pcg_iters = it;
        a.stats->pcg_res0 = (double)res0;
        a.stats->pcg_res = sqrt(A::to_double(rr2s));
    }
}

template <typename DT, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_pcg(PcgArgs a)
{
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
                               const ed_solver_params *prm, ed_stats *stats, PcgArgs &a)
{
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
    a.z = ctx->vec + 2 * P;
    a.p0 = ctx->vec + 3 * P;
    a.p1 = ctx->vec + 4 * P;
    a.part = ctx->pcg_part;
    a.bar = (unsigned *)(ctx->misc + MI_BAR);
    a.status = ctx->misc + MI_STATUS;
    a.stats = stats;
    // every vector is read as float4 rows: 16-byte alignment is required
    const float *vv[4] = {a.d, a.z, a.p0, a.p1};
    for (int i = 0; i < 4; ++i)
        if ((uintptr_t)vv[i] & 15) return ED_ERR_STATE;
    if (((uintptr_t)a.bsr & 15) || ((uintptr_t)a.minv & 15)) return ED_ERR_STATE;
    return ED_OK;
}

static cudaError_t launch_coop(const void *fn, int grid, int nt, void **args, size_t smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

ed_status ed_pcg_solve(ed_context *ctx, const ed_solver_params *prm, ed_stats *stats, cudaStream_t st)
{
    const bool mixed = prm->precision == ED_PRECISION_MIXED;
    if (ctx->pcg.grid <= 0) return ED_ERR_STATE;
    PcgArgs a;
    ed_status s = pcg_fill_args(ctx, ctx->pcg, ctx->pcg_rows, prm, stats, a);
    if (s != ED_OK) return s;
    ED_CUDA_TRY(cudaMemsetAsync(ctx->misc + MI_BAR, 0, 2 * sizeof(int), st));
    void *args[] = {&a};
    ed_tm_begin(ctx, ED_KERNEL_PCG, st);
    ed_note_launch();
    const void *fn = mixed ? (const void *)k_pcg<double, 512> : (const void *)k_pcg<float, 512>;
    cudaError_t e = launch_coop(fn, ctx->pcg.grid, 512, args, ctx->pcg.smem, st);
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
        if (!c->have_graph) return ED_ERR_STATE;
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
                             ed_stats *const *stats, cudaStream_t st)
{
    const int count = bp->count;
    const bool mixed = prm[0]->precision == ED_PRECISION_MIXED;
    PcgBatchParams b;
    memset(&b, 0, sizeof(b));
    b.count = count;
    for (int p = 0; p <= count; ++p) b.cta_first[p] = bp->cta_first[p];
    for (int p = 0; p < count; ++p) {
        if ((prm[p]->precision == ED_PRECISION_MIXED) != mixed) return ED_ERR_ARG;
        ed_status s = pcg_fill_args(ctxs[p], bp->plan[p], ctxs[p]->pcg_rows_b, prm[p], stats[p], b.probs[p]);
        if (s != ED_OK) return s;
        ED_CUDA_TRY(cudaMemsetAsync(ctxs[p]->misc + MI_BAR, 0, 2 * sizeof(int), st));
    }
    void *args[] = {&b};
    const void *fn;
    if (bp->nt == 512) fn = mixed ? (const void *)k_pcg_batch<double, 512> : (const void *)k_pcg_batch<float, 512>;
    else fn = mixed ? (const void *)k_pcg_batch<double, 256> : (const void *)k_pcg_batch<float, 256>;
    ed_note_launch();
    cudaError_t e = launch_coop(fn, bp->grid, bp->nt, args, bp->smem, st);
    if (e != cudaSuccess) {
        fprintf(stderr, "libed: batched PCG launch failed: %s\n", cudaGetErrorString(e));
        return ED_ERR_CUDA;
    }
    return ED_OK;
}
