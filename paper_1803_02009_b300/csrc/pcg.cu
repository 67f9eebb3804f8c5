// pcg.cu -- block-Jacobi preconditioned conjugate gradients on the normal
// equations of one Gauss-Newton step (Sec. II.F), as one persistent
// cooperative kernel.
//
// Layout: H is a symmetric block-sparse matrix over the m nodes (12x12
// blocks, both triangles stored, row-major blocks) bordered by the 6 pose
// unknowns: pose-node blocks C_j (6x12) and a 6x6 pose block.  Every CTA owns
// a contiguous range of node rows; CTA 0 also owns the pose rows.  One PCG
// iteration needs two grid-wide barriers: after q = H p (to reduce p^T q and
// the pose row) and after the preconditioner (to reduce r^T z).  The search
// direction p_k = z_k + beta p_{k-1} is formed on the fly for every block
// column read by the product, so p needs no third barrier (double buffer).
// All reductions are per-CTA partials summed in CTA order by every CTA:
// deterministic.  Every barrier wait is bounded (ED_ERR_TIMEOUT).
#include "ed_internal.cuh"

#define PCG_T 512
#define ROWS_PER_PASS (PCG_T / 36)
#define BAR_TIMEOUT_NS 2000000000ull

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid barrier with a monotonic arrival counter; returns false when the
// context status is set (error elsewhere or timeout)
__device__ bool grid_sync(unsigned *count, unsigned *gen, int *status, unsigned nblocks, unsigned &target,
                          int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += 1;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u) + 1u;
        if (arrived == nblocks * target) {
            __threadfence();
            atomicExch(gen, target);
        } else {
            const unsigned long long t0 = gtimer();
            while (ld_acquire(gen) < target) {
                if (*(volatile int *)status != ED_OK) { ok = 0; break; }
                if (gtimer() - t0 > BAR_TIMEOUT_NS) {
                    atomicCAS(status, ED_OK, ED_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        if (*(volatile int *)status != ED_OK) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

struct PcgArgs {
    int m, n_iter;
    float tol;
    const int *row_ptr, *col;
    const float *bsr, *pnode, *minv, *pose_blk, *grad;
    float *d, *r, *z, *p0, *p1, *q;
    double *part;        // [2][grid][ED_PCG_PART]
    unsigned *bar;       // count, generation
    int *status;
    ed_stats *stats;
};

// sums component k of all CTA partials (warp k: lanes stride over the CTAs in
// a fixed order, then a fixed shuffle tree) -- every CTA gets the same result
template <typename DT>
__device__ __forceinline__ void sum_partials(const double *part, int nb, int ncomp, DT *out_sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < ncomp) {
        DT s = 0;
#pragma unroll 4
        for (int c = lane; c < nb; c += 32) s += (DT)__ldcg(part + c * ED_PCG_PART + w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out_sh[w] = s;
    }
    __syncthreads();
}

// block reduction of NV values per thread; result in sh_out[0..NV) (all threads)
template <typename DT, int NV>
__device__ __forceinline__ void block_sum_n(DT (&v)[NV], DT (*sh)[8], DT *sh_out)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        DT x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        DT s = 0;
        for (int w = 0; w < PCG_T / 32; ++w) s += sh[w][threadIdx.x];
        sh_out[threadIdx.x] = s;
    }
    __syncthreads();
}

template <typename DT>
__global__ void __launch_bounds__(PCG_T) k_pcg(PcgArgs a)
{
    __shared__ int s_flag;
    __shared__ DT s_red[PCG_T / 32][8];
    __shared__ DT s_sum[8];
    __shared__ DT s_blk[8];
    __shared__ float s_pp[6], s_ppold[6], s_qp[6];
    __shared__ DT s_rho, s_beta, s_rr, s_res0;
    const unsigned nb = gridDim.x;
    unsigned target = 0;
    const int m = a.m;
    const int rows_per = (m + nb - 1) / nb;
    const int r0 = min(m, (int)blockIdx.x * rows_per), r1 = min(m, r0 + rows_per);
    const int t = threadIdx.x;
    const int grp = t / 36, tr = t % 36, rr = tr / 3, cg = tr % 3;
    const bool in_grp = grp < ROWS_PER_PASS;
    const int P = 12 * m;
    const float *Hpp = a.pose_blk, *Mp = a.pose_blk + 36;
    double *part0 = a.part, *part1 = a.part + (size_t)ED_MAX_PCG_GRID * ED_PCG_PART;

    if (*(volatile int *)a.status != ED_OK) return;

    // ---- setup: d = 0, r = b = -J^T r, z = M^-1 r ----
    DT rz = 0, rrs = 0;
    for (int j0 = r0; j0 < r1; j0 += ROWS_PER_PASS) {
        const int j = j0 + grp;
        const bool act = in_grp && j < r1;
        float zp = 0.f;
        if (act) {
            // z_j = Minv_j b_j: thread (rr, cg) does row rr, columns 4cg..4cg+3
            const float4 mv = *reinterpret_cast<const float4 *>(a.minv + (size_t)j * 144 + rr * 12 + 4 * cg);
            const float *gj = a.grad + 12 * j + 4 * cg;
            zp = -(mv.x * gj[0] + mv.y * gj[1] + mv.z * gj[2] + mv.w * gj[3]);
        }
        __shared__ float s_z[ROWS_PER_PASS][12][3];
        if (in_grp) s_z[grp][rr][cg] = zp;
        __syncthreads();
        if (act && cg == 0) {
            const float zz = s_z[grp][rr][0] + s_z[grp][rr][1] + s_z[grp][rr][2];
            const float bb = -a.grad[12 * j + rr];
            a.r[12 * j + rr] = bb;
            a.z[12 * j + rr] = zz;
            a.d[12 * j + rr] = 0.f;
            rz += (DT)bb * (DT)zz;
            rrs += (DT)bb * (DT)bb;
        }
        __syncthreads();
    }
    {
        DT vv[2] = {rz, rrs};
        block_sum_n<DT, 2>(vv, s_red, s_blk);
    }
    if (t == 0) {
        DT v1 = s_blk[0], v2 = s_blk[1];
        if (blockIdx.x == 0) {
            DT rzp = 0, rrp = 0;
            for (int i = 0; i < 6; ++i) {
                const float bi = -a.grad[P + i];
                float zi = 0.f;
                for (int k = 0; k < 6; ++k) zi += Mp[6 * i + k] * -a.grad[P + k];
                a.r[P + i] = bi;
                a.z[P + i] = zi;
                a.d[P + i] = 0.f;
                rzp += (DT)bi * (DT)zi;
                rrp += (DT)bi * (DT)bi;
            }
            v1 += rzp;
            v2 += rrp;
        }
        part0[blockIdx.x * ED_PCG_PART + 0] = (double)v1;
        part0[blockIdx.x * ED_PCG_PART + 1] = (double)v2;
    }
    if (!grid_sync(a.bar, a.bar + 1, a.status, nb, target, &s_flag)) return;
    sum_partials<DT>(part0, nb, 2, s_sum);
    if (t == 0) {
        s_rho = s_sum[0];
        s_rr = s_sum[1];
        s_res0 = sqrt((double)s_sum[1]);
        s_beta = 0;
    }
    if (t < 6) s_ppold[t] = 0.f;
    __syncthreads();

    int it = 0;
    for (; it < a.n_iter; ++it) {
        const DT rho = s_rho;
        if (!(rho > (DT)0)) break;
        if (a.tol > 0.f && sqrt((double)s_rr) <= (double)a.tol * (double)s_res0) break;
        const float beta = (float)s_beta;
        const float *pold = (it & 1) ? a.p0 : a.p1;
        float *pnew = (it & 1) ? a.p1 : a.p0;
        // pose part of p: p_pose = z_pose + beta p_pose_old (every CTA)
        if (t < 6) s_pp[t] = __ldcg(a.z + P + t) + beta * s_ppold[t];
        __syncthreads();
        // ---- phase A: q = H p over own rows; partials p.q and C p ----
        DT pq = 0;
        DT cp[6] = {0, 0, 0, 0, 0, 0};
        for (int j0 = r0; j0 < r1; j0 += ROWS_PER_PASS) {
            const int j = j0 + grp;
            const bool act = in_grp && j < r1;
            float acc = 0.f;
            if (act) {
                const int b0 = a.row_ptr[j], b1 = a.row_ptr[j + 1];
                for (int bk = b0; bk < b1; ++bk) {
                    const int l = a.col[bk];
                    const float4 h = __ldg(reinterpret_cast<const float4 *>(a.bsr + (size_t)bk * 144 + rr * 12 + 4 * cg));
                    const float4 zl = __ldcg(reinterpret_cast<const float4 *>(a.z + 12 * l + 4 * cg));
                    float4 pl = zl;
                    if (it > 0) {
                        const float4 po = __ldcg(reinterpret_cast<const float4 *>(pold + 12 * l + 4 * cg));
                        pl = make_float4(zl.x + beta * po.x, zl.y + beta * po.y, zl.z + beta * po.z, zl.w + beta * po.w);
                    }
                    acc += h.x * pl.x + h.y * pl.y + h.z * pl.z + h.w * pl.w;
                }
                if (cg == 0) {
                    const float *C = a.pnode + (size_t)j * 72;
#pragma unroll
                    for (int s = 0; s < 6; ++s) acc += C[12 * s + rr] * s_pp[s];
                }
            }
            __shared__ float s_q[ROWS_PER_PASS][12][3];
            if (in_grp) s_q[grp][rr][cg] = acc;
            __syncthreads();
            if (act && cg == 0) {
                const float qv = s_q[grp][rr][0] + s_q[grp][rr][1] + s_q[grp][rr][2];
                const int e = 12 * j + rr;
                float pv = __ldcg(a.z + e);
                if (it > 0) pv += beta * __ldcg(pold + e);
                pnew[e] = pv;
                a.q[e] = qv;
                pq += (DT)pv * (DT)qv;
                const float *C = a.pnode + (size_t)j * 72;
#pragma unroll
                for (int s = 0; s < 6; ++s) cp[s] += (DT)C[12 * s + rr] * (DT)pv;
            }
            __syncthreads();
        }
        {
            DT vv[7] = {pq, cp[0], cp[1], cp[2], cp[3], cp[4], cp[5]};
            block_sum_n<DT, 7>(vv, s_red, s_blk);
            if (t < 7) part1[blockIdx.x * ED_PCG_PART + t] = (double)s_blk[t];
        }
        if (!grid_sync(a.bar, a.bar + 1, a.status, nb, target, &s_flag)) return;
        // ---- phase B: alpha, d += alpha p, r -= alpha q, z = M^-1 r ----
        sum_partials<DT>(part1, nb, 7, s_sum);
        __shared__ DT s_alpha;
        __shared__ int s_break;
        if (t == 0) {
            DT pqt = s_sum[0];
            for (int i = 0; i < 6; ++i) {
                float qi = 0.f;
                for (int k = 0; k < 6; ++k) qi += Hpp[6 * i + k] * s_pp[k];
                qi += (float)s_sum[1 + i];
                s_qp[i] = qi;
                pqt += (DT)s_pp[i] * (DT)qi;
            }
            s_break = !(pqt > (DT)0);
            s_alpha = rho / pqt;
            if (s_break && blockIdx.x == 0) atomicCAS(a.status, ED_OK, ED_ERR_BREAKDOWN);
        }
        __syncthreads();
        if (s_break) break;
        const float alpha = (float)s_alpha;
        for (int e = 12 * r0 + t; e < 12 * r1; e += PCG_T) {
            const float pv = pnew[e];
            a.d[e] += alpha * pv;
            a.r[e] -= alpha * a.q[e];
        }
        __syncthreads();
        DT rz2 = 0, rr2 = 0;
        for (int j0 = r0; j0 < r1; j0 += ROWS_PER_PASS) {
            const int j = j0 + grp;
            const bool act = in_grp && j < r1;
            float zp = 0.f;
            if (act) {
                const float4 mv = *reinterpret_cast<const float4 *>(a.minv + (size_t)j * 144 + rr * 12 + 4 * cg);
                const float4 rv = *reinterpret_cast<const float4 *>(a.r + 12 * j + 4 * cg);
                zp = mv.x * rv.x + mv.y * rv.y + mv.z * rv.z + mv.w * rv.w;
            }
            __shared__ float s_z2[ROWS_PER_PASS][12][3];
            if (in_grp) s_z2[grp][rr][cg] = zp;
            __syncthreads();
            if (act && cg == 0) {
                const float zz = s_z2[grp][rr][0] + s_z2[grp][rr][1] + s_z2[grp][rr][2];
                const float rv = a.r[12 * j + rr];
                a.z[12 * j + rr] = zz;
                rz2 += (DT)rv * (DT)zz;
                rr2 += (DT)rv * (DT)rv;
            }
            __syncthreads();
        }
        {
            DT vv[2] = {rz2, rr2};
            block_sum_n<DT, 2>(vv, s_red, s_blk);
        }
        if (t == 0) {
            DT w1 = s_blk[0], w2 = s_blk[1];
            if (blockIdx.x == 0) {
                float rp[6];
                for (int i = 0; i < 6; ++i) {
                    a.d[P + i] += alpha * s_pp[i];
                    rp[i] = a.r[P + i] - alpha * s_qp[i];
                    a.r[P + i] = rp[i];
                }
                for (int i = 0; i < 6; ++i) {
                    float zi = 0.f;
                    for (int k = 0; k < 6; ++k) zi += Mp[6 * i + k] * rp[k];
                    a.z[P + i] = zi;
                    w1 += (DT)rp[i] * (DT)zi;
                    w2 += (DT)rp[i] * (DT)rp[i];
                }
            }
            part0[blockIdx.x * ED_PCG_PART + 0] = (double)w1;
            part0[blockIdx.x * ED_PCG_PART + 1] = (double)w2;
        }
        if (!grid_sync(a.bar, a.bar + 1, a.status, nb, target, &s_flag)) return;
        sum_partials<DT>(part0, nb, 2, s_sum);
        if (t == 0) {
            s_beta = s_sum[0] / rho;
            s_rho = s_sum[0];
            s_rr = s_sum[1];
        }
        if (t < 6) s_ppold[t] = s_pp[t];
        __syncthreads();
    }
    if (blockIdx.x == 0 && t == 0 && a.stats) {
        a.stats->pcg_iters = it;
        a.stats->pcg_res0 = (double)s_res0;
        a.stats->pcg_res = sqrt((double)s_rr);
    }
}

ed_status ed_pcg_solve(ed_context *ctx, const ed_solver_params *prm, ed_stats *stats, cudaStream_t st)
{
    const int m = ctx->m;
    const size_t P = ctx->vec_stride;
    const bool mixed = prm->precision == ED_PRECISION_MIXED;
    if (ctx->pcg_grid == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg<double>, PCG_T, 0) != cudaSuccess || occ < 1)
            return ED_ERR_CUDA;
        int occ2 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_pcg<float>, PCG_T, 0) != cudaSuccess || occ2 < 1)
            return ED_ERR_CUDA;
        if (occ2 < occ) occ = occ2;
        int g = ctx->num_sms;   // one CTA per SM: fewest barrier arrivals
        if (g > ED_MAX_PCG_GRID) g = ED_MAX_PCG_GRID;
        ctx->pcg_grid = g;
    }
    // fewer CTAs than rows is fine; more CTAs than rows leaves some idle
    int grid = ctx->pcg_grid;
    const int rows_needed = ed_div_up(m, 1);
    if (grid > rows_needed) grid = rows_needed;
    PcgArgs a;
    a.m = m;
    a.n_iter = prm->n_pcg;
    a.tol = prm->pcg_tol;
    a.row_ptr = ctx->row_ptr;
    a.col = ctx->col;
    a.bsr = ctx->bsr;
    a.pnode = ctx->pnode;
    a.minv = ctx->minv;
    a.pose_blk = ctx->pose_blk;
    a.grad = ctx->grad;
    a.d = ctx->vec;
    a.r = ctx->vec + P;
    a.z = ctx->vec + 2 * P;
    a.p0 = ctx->vec + 3 * P;
    a.p1 = ctx->vec + 4 * P;
    a.q = ctx->vec + 5 * P;
    a.part = ctx->pcg_part;
    a.bar = (unsigned *)(ctx->misc + MI_BAR);
    a.status = ctx->misc + MI_STATUS;
    a.stats = stats;
    // every vector is read as float4 rows: 16-byte alignment is required
    const float *vv[6] = {a.d, a.r, a.z, a.p0, a.p1, a.q};
    for (int i = 0; i < 6; ++i)
        if ((uintptr_t)vv[i] & 15) return ED_ERR_STATE;
    if (((uintptr_t)a.bsr & 15) || ((uintptr_t)a.minv & 15)) return ED_ERR_STATE;
    ED_CUDA_TRY(cudaMemsetAsync(ctx->misc + MI_BAR, 0, 2 * sizeof(int), st));
    void *args[] = {&a};
    ed_tm_begin(ctx, ED_KERNEL_PCG, st);
    ed_note_launch();
    cudaError_t e = mixed ? cudaLaunchCooperativeKernel((const void *)k_pcg<double>, grid, PCG_T, args, 0, st)
                          : cudaLaunchCooperativeKernel((const void *)k_pcg<float>, grid, PCG_T, args, 0, st);
    ed_tm_end(ctx, ED_KERNEL_PCG, st);
    if (e != cudaSuccess) {
        fprintf(stderr, "libed: PCG launch failed: %s\n", cudaGetErrorString(e));
        return ED_ERR_CUDA;
    }
    return ED_OK;
}
