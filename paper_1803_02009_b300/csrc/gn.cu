// gn.cu -- one Gauss-Newton step of Eq. (3) (Sec. II.E-F): point pass,
// normal-equation assembly into 12x12 node blocks, pose finalisation and
// update; the energy of Eq. (3) and its gradient for differentiation.
#include <math.h>
#include <string.h>

#include "ed_internal.cuh"

enum { PASS_STEP = 0, PASS_ENERGY = 1, PASS_GRAD = 2 };

struct PointArgs {
    const float4 *pos, *nrm, *w, *g, *x4;
    const ushort4 *idx;
    const double *pose;
    const float *depth;
    const float4 *nmap;
    ed_intrinsics K;
    int n;
    float eps2, cos_eps_n, sw;
    int mode;
    int recompute_w;   // Gaussian weights recomputed from the node indices (energy / gradient path)
    int m;
    float sigma;
    int n_model;       // rows >= n_model: key points, three rows each (E_corr)
    const float4 *kp_tgt;
    float sw_corr;
    int *pix;          // association (written in STEP / ENERGY, read in GRAD)
    int *status_reset; // the step's device status word, cleared by the first thread (STEP), or NULL
    float4 *rec0, *rec1;
    float2 *part;      // [ED_K1_PART][pstride] float-float partials, component-major
    int pstride;
    float *dbg_wpos, *dbg_wnrm;
    int *dbg_pix;
};

// Per point: Eq. (1) warp, visible-point gate, data residual r = n(u).(v~ - Gamma)
// and its derivative factors; per-CTA sums of E_data, the count, the 6x6 pose
// block and the pose gradient (fixed grid-stride order: deterministic).
__global__ void __launch_bounds__(ED_K1_THREADS, 4) k_points(PointArgs a)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    // a Gauss-Newton step starts with a clear status word: nothing before this
    // kernel's end reads it, and no thread of this kernel writes it otherwise
    if (a.status_reset && blockIdx.x == 0 && threadIdx.x == 0) *a.status_reset = ED_OK;
    __shared__ ed_pose_f P;
    __shared__ float red[ED_K1_THREADS / 32][31];
    if (threadIdx.x == 0) ed_pose_eval(a.pose, P);
    __syncthreads();
    // 0 E_data, 1 count, 2..22 pose block, 23..28 pose gradient, 29 non-finite, 30 E_corr
    float acc[31];
#pragma unroll
    for (int k = 0; k < 31; ++k) acc[k] = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const float4 p = a.pos[i], nr = a.nrm[i];
        const ushort4 id = a.idx[i];
        const float4 wi = a.recompute_w ? ed_gauss_weights(p, id, a.g, a.m, a.sigma) : a.w[i];
        const ed_warped W = ed_warp_point(p, nr, id, wi, a.g, a.x4, P.R, P.T);
        const bool kp = i >= a.n_model;
        // the plane of the residual: target point G and normal tn (the pixel's
        // back-projection and normal, or a key point's target and a camera axis)
        bool valid;
        float G[3];
        float4 tn;
        float sw;
        if (!kp) {
            int q;
            if (a.mode == PASS_GRAD) q = a.pix[i];
            else {
                q = ed_associate(W, a.depth, a.nmap, a.K, a.eps2, a.cos_eps_n);
                a.pix[i] = q;
                if (a.dbg_pix) {
                    a.dbg_pix[i] = q;
                    reinterpret_cast<float4 *>(a.dbg_wpos)[i] = make_float4(W.v.x, W.v.y, W.v.z, p.w);
                    reinterpret_cast<float4 *>(a.dbg_wnrm)[i] = make_float4(W.n.x, W.n.y, W.n.z, nr.w);
                }
            }
            valid = q >= 0;
            if (valid) {
                const int u = q % a.K.width, v = q / a.K.width;
                const float D = __ldg(a.depth + q);
                tn = __ldg(a.nmap + q);
                G[0] = ((float)u - a.K.cx) * D / a.K.fx;
                G[1] = ((float)v - a.K.cy) * D / a.K.fy;
                G[2] = D;
            }
            sw = a.sw;
        } else {
            const int t = i - a.n_model, c = t % 3;
            const float4 T = __ldg(a.kp_tgt + t / 3);
            valid = T.w != 0.f;
            G[0] = T.x;
            G[1] = T.y;
            G[2] = T.z;
            tn = make_float4(c == 0 ? 1.f : 0.f, c == 1 ? 1.f : 0.f, c == 2 ? 1.f : 0.f, 1.f);
            sw = a.sw_corr;
        }
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (valid) {
            const float r = sw * (tn.x * (W.v.x - G[0]) + tn.y * (W.v.y - G[1]) + tn.z * (W.v.z - G[2]));
            const float *R = P.R;
            // R^T n(u), scaled by the residual's sqrt(w)
            const float b0 = sw * (R[0] * tn.x + R[3] * tn.y + R[6] * tn.z);
            const float b1 = sw * (R[1] * tn.x + R[4] * tn.y + R[7] * tn.z);
            const float b2 = sw * (R[2] * tn.x + R[5] * tn.y + R[8] * tn.z);
            float jp[6];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const float *d = P.dR + 9 * t;
                const float e0 = d[0] * W.s.x + d[1] * W.s.y + d[2] * W.s.z;
                const float e1 = d[3] * W.s.x + d[4] * W.s.y + d[5] * W.s.z;
                const float e2 = d[6] * W.s.x + d[7] * W.s.y + d[8] * W.s.z;
                jp[t] = sw * (tn.x * e0 + tn.y * e1 + tn.z * e2);
            }
            jp[3] = sw * tn.x;
            jp[4] = sw * tn.y;
            jp[5] = sw * tn.z;
            r0 = make_float4(b0, b1, b2, r);
            r1 = make_float4(jp[0], jp[1], jp[2], 1.0f);
            if (kp) {
                acc[30] += r * r;
            } else {
                acc[0] += r * r;
                acc[1] += 1.0f;
            }
            int k = 2;
#pragma unroll
            for (int t = 0; t < 6; ++t)
#pragma unroll
                for (int s = t; s < 6; ++s) acc[k++] += jp[t] * jp[s];
#pragma unroll
            for (int t = 0; t < 6; ++t) acc[23 + t] += r * jp[t];
            if (!isfinite(r)) acc[29] += 1.0f;
        }
        if (a.mode != PASS_ENERGY) {
            a.rec0[i] = r0;
            a.rec1[i] = r1;
        }
    }
    // block reduction: for each half of the 31 sums a butterfly over the warp
    // that halves the values a lane carries at every shuffle step (lane bit o
    // keeps the upper or the lower half and receives that half from its
    // partner), so lanes 2k and 2k + 1 end with the half's value k (float);
    // then the warps in order (float-float)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
        float x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = 16 * hf + k < 31 ? acc[16 * hf + k] : 0.f;
#pragma unroll
        for (int lvl = 0; lvl < 4; ++lvl) {
            const int o = 16 >> lvl, n = 8 >> lvl;
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < n; ++j) {
                const float send = up ? x[j] : x[j + n];
                const float keep = up ? x[j + n] : x[j];
                x[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        const float v = x[0] + __shfl_xor_sync(0xffffffffu, x[0], 1);
        const int k = 16 * hf + (lane >> 1);
        if (!(lane & 1) && k < 31) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 31) {
        float2 s = make_float2(0.f, 0.f);
        for (int w = 0; w < ED_K1_THREADS / 32; ++w) s = ed_ff_add1(s, red[w][threadIdx.x]);
        a.part[(size_t)threadIdx.x * a.pstride + blockIdx.x] = s;
    }
}

static int k1_grid(const ed_context *ctx)
{
    int g = ed_div_up(ctx->N, ED_K1_THREADS);
    const int cap = 4 * ctx->num_sms;
    if (g > cap) g = cap;
    if (g > ctx->max_k1_ctas) g = ctx->max_k1_ctas;
    return g < 1 ? 1 : g;
}

ed_status ed_point_pass(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, const float *x,
                        const double *pose, int mode, cudaStream_t st)
{
    PointArgs a;
    a.pos = (const float4 *)ctx->pos;
    a.nrm = (const float4 *)ctx->nrm;
    a.w = (const float4 *)ctx->graph.weights;
    a.g = (const float4 *)ctx->graph.nodes;
    a.x4 = (const float4 *)x;
    a.idx = (const ushort4 *)ctx->graph.idx;
    a.pose = pose;
    a.depth = fr->depth;
    a.nmap = (const float4 *)fr->nmap;
    a.K = fr->intr;
    a.n = ctx->N;
    a.eps2 = prm->eps_d * prm->eps_d;
    a.cos_eps_n = prm->cos_eps_n;
    a.sw = sqrtf(prm->w_data);
    a.mode = mode;
    // the autograd path (energy, gradient) recomputes Gaussian skinning
    // weights instead of reading the stored ones (bit-identical values)
    a.recompute_w = mode != PASS_STEP && ctx->weight_mode == ED_WEIGHT_GAUSSIAN;
    a.m = ctx->m;
    a.sigma = ctx->sigma;
    a.n_model = ctx->n_kp > 0 ? ctx->n_model : ctx->N;
    a.kp_tgt = ctx->kp_tgt;
    a.sw_corr = sqrtf(ctx->w_corr);
    a.pix = ctx->pix;
    a.status_reset = mode == PASS_STEP ? ctx->misc + MI_STATUS : nullptr;
    a.rec0 = mode == PASS_GRAD ? ctx->gpts : ctx->rec0;
    a.rec1 = mode == PASS_GRAD ? ctx->gpts + ctx->lim.max_points : ctx->rec1;
    a.part = ctx->k1_part;
    a.pstride = ctx->max_k1_ctas;
    a.dbg_wpos = ctx->dbg_wpos;
    a.dbg_wnrm = ctx->dbg_wnrm;
    a.dbg_pix = (mode == PASS_STEP && ctx->dbg_wpos && ctx->dbg_wnrm) ? ctx->dbg_pix : nullptr;
    if (mode == PASS_STEP) ed_tm_begin(ctx, ED_KERNEL_POINTS, st);
    ED_CUDA_TRY(ed_launch_pdl(k_points, dim3(k1_grid(ctx)), dim3(ED_K1_THREADS), 0, st, a)); ed_note_launch();
    if (mode == PASS_STEP) ed_tm_end(ctx, ED_KERNEL_POINTS, st);
    ED_LAUNCH_CHECK();
    return ED_OK;
}

// ---------------------------------------------------------------------------
// assembly: one warp per chunk of <= ED_CHUNK entries of one upper block (j, l)
// role 0: the 60 independent entries of sum c (nb nb^T) (x) (d^ d^T),
//         d^ = [v - g_j; 1], c = w_s w_t  (every data-term block of J^T J)
// role 1 (diagonal blocks): J^T r (12) and the pose-node block (6 x 12)
// The per-entry geometry (d, c) was written at graph build; the residual
// record of the point is gathered (entries of a chunk are in point order).
// ---------------------------------------------------------------------------

// Recursive halving of NV float2 values per lane across the warp (fixed order,
// so the result is deterministic): after the step with offset o every lane
// keeps the half selected by bit o of its lane index and adds the partner's
// copy of it.  At the end lane k holds the sums of float2 values
// (NV/32) k ... (NV/32) k + NV/32 - 1.
template <int NV>
__device__ __forceinline__ void warp_halving2(float2 (&v)[NV])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, n = NV; o > 0; o >>= 1, n >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < n / 2; ++k) {
            const float2 keep = hi ? v[k + n / 2] : v[k];
            const float2 give = hi ? v[k] : v[k + n / 2];
            float2 recv;
            recv.x = __shfl_xor_sync(0xffffffffu, give.x, o);
            recv.y = __shfl_xor_sync(0xffffffffu, give.y, o);
            v[k] = __fadd2_rn(keep, recv);
        }
    }
}

static_assert(ED_CHUNK == 128 && ED_CHUNK1 % 128 == 0, "the assembly kernels take 4 entries per lane (and round)");

// Recursive halving of 16 float2 values per lane down to one per lane pair,
// then the pair: afterwards lanes 2k and 2k + 1 both hold the full sum of
// slot k (fixed order: deterministic).
__device__ __forceinline__ void warp_halving2_16(float2 (&v)[16])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, n = 16; o > 1; o >>= 1, n >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < n / 2; ++k) {
            const float2 keep = hi ? v[k + n / 2] : v[k];
            const float2 give = hi ? v[k] : v[k + n / 2];
            float2 recv;
            recv.x = __shfl_xor_sync(0xffffffffu, give.x, o);
            recv.y = __shfl_xor_sync(0xffffffffu, give.y, o);
            v[k] = __fadd2_rn(keep, recv);
        }
    }
    float2 recv;
    recv.x = __shfl_xor_sync(0xffffffffu, v[0].x, 1);
    recv.y = __shfl_xor_sync(0xffffffffu, v[0].y, 1);
    v[0] = __fadd2_rn(v[0], recv);
}

// role 0: two warps per chunk of <= 128 entries of one upper block (j, l).
// Lane k takes entries k, k + 32, k + 64, k + 96; warp half h forms the 30
// moments c nn_a (d^ d^T)_q of a = 3h .. 3h + 2 (nn = the 6 products of
// n~ = sqrt(w) R^T n, d^ = [v - g_j; 1], paired FP32 FMA), the warp then sums
// them by recursive halving; half h writes moment pairs 15h .. 15h + 14.
__global__ void __launch_bounds__(128) k_assemble0(const int4 *__restrict__ chunks, int nchunks, int max_chunks,
                                                   const float4 *__restrict__ geo, const uint32_t *__restrict__ ent,
                                                   const float4 *__restrict__ rec0, float *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int c = wg >> 1, h = wg & 1;
    if (c >= nchunks) return;
    // the chunk, its geometry and its entries are fixed for the frame: loaded
    // before the wait for the point pass (whose residual records come after)
    const int4 ch = chunks[c];
    float4 gd[4], b[4];
    int pt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = lane + 32 * q;
        gd[q] = e < ch.z ? __ldg(geo + ch.y + e) : make_float4(0.f, 0.f, 0.f, 0.f);   // w = 0: no contribution
        pt[q] = e < ch.z ? (int)(__ldg(ent + ch.y + e) >> 4) : -1;
    }
    ed_pdl_wait();
    ed_pdl_trigger();
    // (the point pass may still have been writing the records while this kernel
    // was alive: coherent loads, not the read-only path)
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = pt[q] >= 0 ? __ldcg(rec0 + pt[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float cf = gd[q].w;
        const float d0 = gd[q].x, d1 = gd[q].y, d2 = gd[q].z;
        // this half's three products: (x x, x y, x z) or (y y, y z, z z), times c
        const float s0 = cf * (h ? b[q].y : b[q].x);
        const float s2 = cf * (h ? b[q].z : b[q].x);
        const float nn[3] = {s0 * (h ? b[q].y : b[q].x), s0 * (h ? b[q].z : b[q].y), s2 * b[q].z};
        // d^ d^T upper triangle in pairs: (d0 d0, d0 d1) (d0 d2, d0) (d1 d1, d1 d2) (d1, d2 d2) (d2, 1)
        const float2 dd[5] = {make_float2(d0 * d0, d0 * d1), make_float2(d0 * d2, d0), make_float2(d1 * d1, d1 * d2),
                              make_float2(d1, d2 * d2), make_float2(d2, 1.0f)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float2 na = make_float2(nn[a], nn[a]);
#pragma unroll
            for (int k = 0; k < 5; ++k) v[5 * a + k] = __ffma2_rn(na, dd[k], v[5 * a + k]);
        }
    }
    warp_halving2_16(v);
    if (!(lane & 1) && (lane >> 1) < 15)   // chunk-major partials: moment pairs 15 h + lane / 2
        reinterpret_cast<float2 *>(part + (long)c * ED_PART_STRIDE)[15 * h + (lane >> 1)] = v[0];
}

// role 1 (diagonal blocks): two warps per chunk of <= ED_CHUNK1 entries (most
// nodes have one chunk), in rounds of 128 entries; per entry J^T r (12 floats)
// and the pose-node block (6 x 12) of node j.  Moment pairs (float2 slots):
// 0..5 J^T r, 6 + 6 t + 2 r (+1) pose-node row t, node row r.  Half 0 forms
// slots 0..23 (J^T r, rows t = 0..2), half 1 slots 24..41 (t = 3..5); the
// loads of two entries are issued together.
template <int H>
__device__ __forceinline__ void assemble1_half(const int4 ch, int c, const float *R, const float4 *__restrict__ geo,
                                               const uint32_t *__restrict__ ent, const float4 *__restrict__ rec0,
                                               const float4 *__restrict__ rec1, float *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    constexpr int BASE = H == 0 ? 6 : 0;   // slot of row t = 3H within this half
    float2 v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int e0 = 0; e0 < ch.z; e0 += 128) {
#pragma unroll
    for (int q0 = 0; q0 < 4; q0 += 2) {
        float4 gd[2], b[2], jq[2];
        int pi[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = e0 + lane + 32 * (q0 + u);
            const bool in = e < ch.z;
            gd[u] = in ? __ldg(geo + ch.y + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            pi[u] = in ? (int)(__ldg(ent + ch.y + e) >> 4) : -1;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            b[u] = pi[u] >= 0 ? __ldg(rec0 + pi[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (H == 0) jq[u] = pi[u] >= 0 ? __ldg(rec1 + pi[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float ws = sqrtf(gd[u].w);   // diagonal entries store w_s * w_s (0 for absent entries)
            const float2 dlo = make_float2(gd[u].x, gd[u].y), dhi = make_float2(gd[u].z, 1.0f);
            const float nb[3] = {ws * b[u].x, ws * b[u].y, ws * b[u].z};
            // d r / d pose: angles (t = 0..2) from the point record, translation
            // (t = 3..5) = R nb_s with nb_s = sqrt(w) R^T n
            float jp[3];
            if (H == 0) {
                jp[0] = jq[u].x;
                jp[1] = jq[u].y;
                jp[2] = jq[u].z;
            } else {
                jp[0] = R[0] * b[u].x + R[1] * b[u].y + R[2] * b[u].z;
                jp[1] = R[3] * b[u].x + R[4] * b[u].y + R[5] * b[u].z;
                jp[2] = R[6] * b[u].x + R[7] * b[u].y + R[8] * b[u].z;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (H == 0) {
                    const float2 g2 = make_float2(b[u].w * nb[r], b[u].w * nb[r]);
                    v[2 * r] = __ffma2_rn(g2, dlo, v[2 * r]);
                    v[2 * r + 1] = __ffma2_rn(g2, dhi, v[2 * r + 1]);
                }
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const float s2 = jp[t] * nb[r];
                    const float2 c2 = make_float2(s2, s2);
                    v[BASE + 6 * t + 2 * r] = __ffma2_rn(c2, dlo, v[BASE + 6 * t + 2 * r]);
                    v[BASE + 6 * t + 2 * r + 1] = __ffma2_rn(c2, dhi, v[BASE + 6 * t + 2 * r + 1]);
                }
            }
        }
    }
    }
    warp_halving2<32>(v);
    constexpr int NSLOT = H == 0 ? 24 : 18;
    if (lane < NSLOT) reinterpret_cast<float2 *>(part + (long)c * ED_PART_STRIDE)[24 * H + lane] = v[0];
}

__global__ void __launch_bounds__(128, 4) k_assemble1(const int4 *__restrict__ chunks, int c_begin, int nchunks,
                                                   int max_chunks, const float4 *__restrict__ geo,
                                                   const uint32_t *__restrict__ ent, const float4 *__restrict__ rec0,
                                                   const float4 *__restrict__ rec1, const double *__restrict__ pose,
                                                   float *__restrict__ part)
{
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int c = c_begin + (wg >> 1), h = wg & 1;
    const int4 ch = c < c_begin + nchunks ? chunks[c] : make_int4(0, 0, 0, 0);   // fixed for the frame
    ed_pdl_wait();
    __shared__ ed_pose_f P;
    if (threadIdx.x == 0) ed_pose_eval(pose, P);
    __syncthreads();
    if (c >= c_begin + nchunks) return;
    if (h == 0) assemble1_half<0>(ch, c, P.R, geo, ent, rec0, rec1, part);
    else assemble1_half<1>(ch, c, P.R, geo, ent, rec0, rec1, part);
}

// ---------------------------------------------------------------------------
// finalisation: one warp per upper block (j, l), j <= l
// ---------------------------------------------------------------------------

struct FinArgs {
    const int4 *info;        // [n_upper][2] records of the upper blocks (k_fin_pack)
    const int *col, *nbr;
    const float *part;
    int max_chunks;
    int n_upper, kg, mixed;
    const float4 *g;
    const float4 *x4;
    float w_rot, w_reg, lambda, jitter;
    float *bsr, *grad, *pnode, *minv;
    float2 *node_energy;
    int *status;
    // for k_fin_totals: the energy totals of the step from the node energies
    // and the pose pass's sums
    int m;
    int *misc;
    double *dmisc;
    ed_stats *stats;
    float lambda_report;     // damping reported in the statistics
};

__device__ __forceinline__ int sym3(int a, int b)
{
    if (a > b) { int t = a; a = b; b = t; }
    return a == 0 ? b : (a == 1 ? 2 + b : 5);
}
__device__ __forceinline__ int sym4(int a, int b)
{
    if (a > b) { int t = a; a = b; b = t; }
    return a == 0 ? b : (a == 1 ? 3 + b : (a == 2 ? 5 + b : 9));
}

// sum of the chunk partials of one component (partials are chunk-major,
// ED_PART_STRIDE floats per chunk): p = the component in the first chunk
// (NULL: none), n chunks, summed in chunk order, two-sum compensated when
// mixed.  A lane keeps several of them and loads four chunks of each before
// adding, so the loads of all its components are in flight together.
struct PartSum {
    const float *p;
    int n;
    float s, err;
};

__device__ __forceinline__ PartSum part_sum(const float *part, int comp, int c0, int n)
{
    PartSum r;
    r.p = comp >= 0 ? part + (long)c0 * ED_PART_STRIDE + comp : nullptr;
    r.n = comp >= 0 ? n : 0;
    r.s = 0.f;
    r.err = 0.f;
    return r;
}

__device__ __forceinline__ void part_load4(const PartSum &c, int k0, float4 &v)
{
    const float *p = c.p + (long)k0 * ED_PART_STRIDE;
    v.x = k0 < c.n ? p[0] : 0.f;
    v.y = k0 + 1 < c.n ? p[ED_PART_STRIDE] : 0.f;
    v.z = k0 + 2 < c.n ? p[2 * ED_PART_STRIDE] : 0.f;
    v.w = k0 + 3 < c.n ? p[3 * ED_PART_STRIDE] : 0.f;
}

__device__ __forceinline__ void part_add1(PartSum &c, float x, bool in, int mixed)
{
    if (!in) return;
    if (!mixed) {
        c.s += x;
        return;
    }
    const float t = c.s + x;
    const float bp = t - c.s;
    c.err += (c.s - (t - bp)) + (x - bp);
    c.s = t;
}

__device__ __forceinline__ void part_add4(PartSum &c, int k0, const float4 v, int mixed)
{
    part_add1(c, v.x, k0 < c.n, mixed);
    part_add1(c, v.y, k0 + 1 < c.n, mixed);
    part_add1(c, v.z, k0 + 2 < c.n, mixed);
    part_add1(c, v.w, k0 + 3 < c.n, mixed);
}

__device__ __forceinline__ float part_value(const PartSum &c, int mixed) { return mixed ? c.s + c.err : c.s; }

// derivative of the Rot(A) residual q (column pair ca, cb) with respect to
// the parameter 4 r + c of [A | t]
__device__ __forceinline__ float rot_jac(const float *X, int q, int r, int c)
{
    const int ca = q < 3 ? (q < 2 ? 0 : 1) : q - 3;
    const int cb = q < 3 ? (q == 0 ? 1 : 2) : q - 3;
    float v = 0.f;
    if (c == ca) v += X[4 * r + cb];
    if (c == cb) v += X[4 * r + ca];
    return v;
}

__device__ __forceinline__ float rot_res(const float *X, int q)
{
    const int ca = q < 3 ? (q < 2 ? 0 : 1) : q - 3;
    const int cb = q < 3 ? (q == 0 ? 1 : 2) : q - 3;
    float d = X[ca] * X[cb] + X[4 + ca] * X[4 + cb] + X[8 + ca] * X[8 + cb];
    return ca == cb ? d - 1.0f : d;
}

#define FIN_WARPS 4

// E_rot Gauss-Newton block between columns c and cp of A (3-vectors x_c over
// node rows r, rp): sum over the 6 residuals x_a.x_b - delta_ab of products of
// their derivatives; c != cp: x_cp[r] x_c[rp]; c == cp: 4 x_c[r] x_c[rp] +
// sum_{d != c} x_d[r] x_d[rp]
__device__ __forceinline__ float rot_jtj(const float *X, int r, int c, int rp, int cp)
{
    if (c != cp) return X[4 * r + cp] * X[4 * rp + c];
    float v = 4.0f * X[4 * r + c] * X[4 * rp + c];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d != c) v += X[4 * r + d] * X[4 * rp + d];
    return v;
}

// block-Jacobi inverse of one 12x12 block H (shared memory, row-major; one
// warp): Gauss-Jordan elimination without pivoting on [H + jitter tr/12 I | I].
// H is symmetric positive definite, so every pivot is positive (the pivots
// are the squares of the Cholesky pivots).  Lane r < 24 keeps row r % 12 of
// the left (r < 12) or the right half in registers; the pivot row and the
// elimination factors travel by shuffles, so the 12 steps have no shared
// memory traffic.  The right half, symmetrised through `scratch` (144
// floats), goes to out (row-major); false, with out untouched, on a
// non-positive pivot.
__device__ __forceinline__ bool block_inverse12(const float *H, float *scratch, float jitter, float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int r = lane < 24 ? lane % 12 : 0, half = lane >= 12 && lane < 24 ? 1 : 0;
    float tr = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) tr += H[k * 13];
    const float jd = jitter * tr / 12.0f;
    float v[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = half ? (c == r ? 1.0f : 0.0f) : H[r * 12 + c] + (c == r ? jd : 0.0f);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float piv = __shfl_sync(0xffffffffu, v[k], k);   // row k, column k (left half)
        const float fr = __shfl_sync(0xffffffffu, v[k], r);    // row r, column k (left half)
        ok = ok && piv > 0.0f;
        const float ip = 1.0f / piv, f = -fr * ip;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const float pc = __shfl_sync(0xffffffffu, v[c], k + 12 * half);   // pivot row, this lane's half
            v[c] = r == k ? pc * ip : fmaf(f, pc, v[c]);
        }
    }
    if (!ok) return false;
    __syncwarp();
    if (half) {
#pragma unroll
        for (int c = 0; c < 12; ++c) scratch[r * 12 + c] = v[c];
    }
    __syncwarp();
    for (int e = lane; e < 144; e += 32) {
        const int p = e / 12, q = e - 12 * p;
        out[e] = 0.5f * (scratch[e] + scratch[q * 12 + p]);
    }
    __syncwarp();
    return true;
}

// the entry table of a 12x12 block: moment index of (R, C) and of (R, 3-column
// shift), R, C
__device__ __forceinline__ void fill_block_table(int *s_tab)
{
    for (int e = threadIdx.x; e < 144; e += blockDim.x) {
        const int R = e / 12, Cc = e % 12;
        const int r = R >> 2, c = R & 3, rp = Cc >> 2, cp = Cc & 3;
        const int mi = 10 * sym3(r, rp) + sym4(c, cp), m3 = 10 * sym3(r, rp) + sym4(c, 3);
        s_tab[e] = mi | (m3 << 8) | (R << 16) | (Cc << 24);
    }
}

// component i of (v0, v1, v2, v3) without a local array
__device__ __forceinline__ float pick4(float v0, float v1, float v2, float v3, int i)
{
    return i == 0 ? v0 : (i == 1 ? v1 : (i == 2 ? v2 : v3));
}

// the partial sums of components (c_a, c_b) over n chunks from c0 (c_b < 0: one)
__device__ __forceinline__ void part_sums2(const FinArgs &a, int ca, int cb, int c0, int n, float &va, float &vb)
{
    PartSum pa = part_sum(a.part, ca, c0, n), pb = part_sum(a.part, cb, c0, n);
    for (int k0 = 0; k0 < pa.n; k0 += 4) {
        float4 x, y;
        part_load4(pa, k0, x);
        part_load4(pb, k0, y);
        part_add4(pa, k0, x, a.mixed);
        part_add4(pb, k0, y, a.mixed);
    }
    va = part_value(pa, a.mixed);
    vb = part_value(pb, a.mixed);
}

// the same for three components (cc < 0: none)
__device__ __forceinline__ void part_sums3(const FinArgs &a, int ca, int cb, int cc, int c0, int n, float &va, float &vb,
                                           float &vc)
{
    PartSum pa = part_sum(a.part, ca, c0, n), pb = part_sum(a.part, cb, c0, n), pc = part_sum(a.part, cc, c0, n);
    for (int k0 = 0; k0 < pa.n; k0 += 4) {
        float4 x, y, z;
        part_load4(pa, k0, x);
        part_load4(pb, k0, y);
        part_load4(pc, k0, z);
        part_add4(pa, k0, x, a.mixed);
        part_add4(pb, k0, y, a.mixed);
        part_add4(pc, k0, z, a.mixed);
    }
    va = part_value(pa, a.mixed);
    vb = part_value(pb, a.mixed);
    vc = part_value(pc, a.mixed);
}

// one warp per upper block u (INV = false: the block inverses are taken
// later, in the Levenberg-Marquardt stage).  The 144 entries of a block go to
// lanes 0..23: lane L takes column C = L % 12 of the rows R = L / 12 + 2 k,
// k < 6, so a lane's column quantities are formed once.
template <bool INV>
__device__ __forceinline__ void finalize_block(const FinArgs &a, int u, float *M, float *H, float *X, float *S,
                                               float *Lw, int *Nk, float4 *Ng, float *Nx, const int *s_tab)
{
    const int lane = threadIdx.x & 31;
    const int4 i0 = a.info[2 * u], i1 = a.info[2 * u + 1];
    const int b = i0.x, j = i0.y, l = i0.z;
    const bool diag = j == l;
    const int c0 = i1.x, nch = i1.y;
    const int Cc = lane % 12, h0 = lane < 12 ? 0 : 1, rp = Cc >> 2, cp = Cc & 3;
    const bool ent_lane = lane < 24;
    const float wr = a.w_reg;
    if (!diag) {
        const int tb = i0.w;
        const bool e_jl = (i1.z & 1) != 0, e_lj = (i1.z & 2) != 0;   // graph edges j -> l, l -> j
        const float4 gj = a.g[j], gl = a.g[l];
        {
            float v0, v1;
            part_sums2(a, lane, lane + 32 < 60 ? lane + 32 : -1, c0, nch, v0, v1);
            M[lane] = v0;
            if (lane + 32 < 60) M[lane + 32] = v1;
        }
        __syncwarp();
        if (tb < 0) {
            if (lane == 0) atomicCAS(a.status, 0, ED_ERR_STATE);
            return;
        }
        if (!ent_lane) return;
        // d^_l = d^_j + [g_j - g_l; 0]; h_jl = [g_l - g_j; 1]
        const float dlc = pick4(gj.x - gl.x, gj.y - gl.y, gj.z - gl.z, 0.f, cp);
        const float hx = gl.x - gj.x, hy = gl.y - gj.y, hz = gl.z - gj.z;
        // E_reg, edge l -> j (d e / d t_j = -I): column quantity of the rows c = 3
        const float reg_lj = e_lj ? -wr * (cp < 3 ? -pick4(hx, hy, hz, 1.f, cp) : 1.0f) : 0.f;
        float *dst = a.bsr + (long)b * 144 + Cc;
        float *dstT = a.bsr + (long)tb * 144 + Cc * 12;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int R = h0 + 2 * k, r = R >> 2, c = R & 3;
            const int T = s_tab[R * 12 + Cc];
            float h = M[T & 255];
            if (cp < 3) h += dlc * M[(T >> 8) & 255];
            if (r == rp) {   // E_reg, edge j -> l (d e / d t_l = -I) on the t column
                if (e_jl && cp == 3) h -= wr * pick4(hx, hy, hz, 1.f, c);
                if (c == 3) h += reg_lj;
            }
            dst[R * 12] = h;
            dstT[R] = h;
        }
        return;
    }
    // ---- diagonal block ----
    const int rp0 = i0.w, rp1 = rp0 + (i1.w >> 16);   // row j of the block pattern
    if (lane < a.kg) {   // out-edges j -> k: index, position and parameters of k, loaded once
        const int k = a.nbr[j * a.kg + lane];
        Nk[lane] = k;
        if (k >= 0) {
            Ng[lane] = a.g[k];
#pragma unroll
            for (int q = 0; q < 3; ++q) reinterpret_cast<float4 *>(Nx + 12 * lane)[q] = a.x4[3 * k + q];
        }
    }
    if (lane < 12) X[lane] = (&a.x4[3 * j].x)[lane];
    const float4 gj = a.g[j];
    // the 60 moments (role-0 chunks), then J^T r and the pose-node block (84
    // components of the role-1 chunks)
    float *Gx = M + 60;
    {
        float v0, v1;
        part_sums2(a, lane, lane + 32 < 60 ? lane + 32 : -1, c0, nch, v0, v1);
        M[lane] = v0;
        if (lane + 32 < 60) M[lane + 32] = v1;
        const int c1 = i1.z, nch1 = i1.w & 0xffff;
        float w0, w1, w2;
        part_sums3(a, lane, lane + 32, lane + 64 < 84 ? lane + 64 : -1, c1, nch1, w0, w1, w2);
        auto put = [&](int k, float v) {
            if (k < 12) Gx[k] = v;
            else a.pnode[(long)j * 72 + (k - 12)] = v;
        };
        put(lane, w0);
        put(lane + 32, w1);
        if (lane + 64 < 84) put(lane + 64, w2);
    }
    __syncwarp();
    // S = sum over out-edges j -> k of h h^T, h = [g_k - g_j; 1]
    if (lane < 16) {
        const int c = lane >> 2, cq = lane & 3;
        float v = 0.f;
        for (int s = 0; s < a.kg; ++s) {
            if (Nk[s] < 0) continue;
            const float4 gk = Ng[s];
            const float hx = gk.x - gj.x, hy = gk.y - gj.y, hz = gk.z - gj.z;
            v += pick4(hx, hy, hz, 1.f, c) * pick4(hx, hy, hz, 1.f, cq);
        }
        S[lane] = v;
    }
    // in-edges k -> j (they lie in row j): count and summed residuals
    float nin = 0.f, ein0 = 0.f, ein1 = 0.f, ein2 = 0.f;
    for (int t = rp0 + lane; t < rp1; t += 32) {
        const int k = a.col[t];
        // the neighbours of k, its position and parameters: every load issued together
        int nb[ED_MAX_KG];
#pragma unroll
        for (int s = 0; s < ED_MAX_KG; ++s) nb[s] = s < a.kg ? a.nbr[k * a.kg + s] : -1;
        const float4 gk = a.g[k];
        const float4 xk0 = a.x4[3 * k], xk1 = a.x4[3 * k + 1], xk2 = a.x4[3 * k + 2];
        bool in = false;
#pragma unroll
        for (int s = 0; s < ED_MAX_KG; ++s) in |= nb[s] == j;
        if (k == j || !in) continue;
        const float hh[3] = {gj.x - gk.x, gj.y - gk.y, gj.z - gk.z};
        const float x0[4] = {xk0.x, xk0.y, xk0.z, xk0.w}, x1[4] = {xk1.x, xk1.y, xk1.z, xk1.w};
        const float x2[4] = {xk2.x, xk2.y, xk2.z, xk2.w};
        nin += 1.f;
        ein0 += ed_reg_residual(x0, 0, hh, X[3]);
        ein1 += ed_reg_residual(x1, 1, hh, X[7]);
        ein2 += ed_reg_residual(x2, 2, hh, X[11]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nin += __shfl_xor_sync(0xffffffffu, nin, o);
        ein0 += __shfl_xor_sync(0xffffffffu, ein0, o);
        ein1 += __shfl_xor_sync(0xffffffffu, ein1, o);
        ein2 += __shfl_xor_sync(0xffffffffu, ein2, o);
    }
    __syncwarp();
    // the 144 entries: data moments + E_rot + E_reg (out-edges S, in-edges on t)
    if (ent_lane) {
        float *dst = a.bsr + (long)b * 144 + Cc;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int R = h0 + 2 * k, r = R >> 2, c = R & 3;
            const int T = s_tab[R * 12 + Cc];
            float h = M[T & 255];
            if (c < 3 && cp < 3) h += a.w_rot * rot_jtj(X, r, c, rp, cp);
            if (r == rp) {
                h += wr * S[4 * c + cp];
                if (c == 3 && cp == 3) h += wr * nin;
            }
            if (R == Cc) h *= 1.0f + a.lambda;   // LM damping
            H[R * 12 + Cc] = h;
            dst[R * 12] = h;
        }
    }
    // gradient: data + E_rot + E_reg (out-edges, in-edges)
    if (lane < 12) {
        const int r = lane >> 2, c = lane & 3;
        float g = Gx[lane];
        if (c < 3) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) v += rot_res(X, q) * rot_jac(X, q, r, c);
            g += a.w_rot * v;
        }
        for (int s = 0; s < a.kg; ++s) {
            if (Nk[s] < 0) continue;
            const float4 gk = Ng[s];
            const float hh[3] = {gk.x - gj.x, gk.y - gj.y, gk.z - gj.z};
            const float er = ed_reg_residual(X + 4 * r, r, hh, Nx[12 * s + 4 * r + 3]);
            g += wr * er * pick4(hh[0], hh[1], hh[2], 1.f, c);
        }
        if (c == 3) g -= wr * (r == 0 ? ein0 : (r == 1 ? ein1 : ein2));
        a.grad[12 * j + lane] = g;
    }
    // energies of node j: Rot(A_j), and its out-edges
    if (lane == 0) {
        float erot = 0.f, ereg = 0.f;
        for (int q = 0; q < 6; ++q) {
            const float rho = rot_res(X, q);
            erot += a.w_rot * rho * rho;
        }
        for (int s = 0; s < a.kg; ++s) {
            if (Nk[s] < 0) continue;
            const float4 gk = Ng[s];
            const float hh[3] = {gk.x - gj.x, gk.y - gj.y, gk.z - gj.z};
            for (int r = 0; r < 3; ++r) {
                const float e = ed_reg_residual(X + 4 * r, r, hh, Nx[12 * s + 4 * r + 3]);
                ereg += wr * e * e;
            }
        }
        a.node_energy[j] = make_float2(erot, ereg);
    }
    __syncwarp();
    if (!INV) return;
    if (!block_inverse12(H, Lw, a.jitter, a.minv + (long)j * 144) && lane == 0)
        atomicCAS(a.status, 0, ED_ERR_BREAKDOWN);
}

// after the finalisation, one CTA: the node energies summed in a fixed order
// (float-float), the energy of Eq. (3) from them and the pose pass's sums,
// the non-finite check, the step's statistics; it also clears the arrival
// count of the step's PCG
__global__ void __launch_bounds__(32 * FIN_WARPS) k_fin_totals(FinArgs a)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    __shared__ float2 s_w[FIN_WARPS][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2 er = make_float2(0.f, 0.f), eg = er;
    for (int j = threadIdx.x; j < a.m; j += 32 * FIN_WARPS) {
        const float2 e = __ldcg(a.node_energy + j);
        er = ed_ff_add1(er, e.x);
        eg = ed_ff_add1(eg, e.y);
    }
    er = ed_ff_warp_sum(er);
    eg = ed_ff_warp_sum(eg);
    if (lane == 0) {
        s_w[w][0] = er;
        s_w[w][1] = eg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 a0 = s_w[0][0], a1 = s_w[0][1];
        for (int k = 1; k < FIN_WARPS; ++k) {
            a0 = ed_ff_add(a0, s_w[k][0]);
            a1 = ed_ff_add(a1, s_w[k][1]);
        }
        const double ne0 = ed_ff_value(a0), ne1 = ed_ff_value(a1);
        const double *ps = a.dmisc + DM_POSE;   // E_data, valid, non-finite flag, E_corr, E_r, E_p
        const double E = ps[0] + ne0 + ne1 + ps[4] + ps[5] + ps[3];
        if (!isfinite(E) || ps[2] > 0.0) atomicCAS(a.status, ED_OK, ED_ERR_NONFINITE);
        a.dmisc[0] = E;
        a.dmisc[1] = ps[0];
        a.dmisc[2] = ne0;
        a.dmisc[3] = ne1;
        a.dmisc[4] = ps[4];
        a.dmisc[5] = ps[5];
        a.dmisc[6] = ps[1];
        a.dmisc[7] = ps[3];
        if (a.stats) {
            a.stats->e_corr = ps[3];
            a.stats->energy = E;
            a.stats->e_data = ps[0];
            a.stats->e_rot = ne0;
            a.stats->e_reg = ne1;
            a.stats->e_rot_prior = ps[4];
            a.stats->e_pos_prior = ps[5];
            a.stats->n_valid = (int)ps[1];
            a.stats->lm_rejected = 0;
            a.stats->lambda = a.lambda_report;
        }
    }
    if (threadIdx.x < 2) a.misc[MI_BAR + threadIdx.x] = 0;   // the arrival count of the step's PCG
}

template <bool INV>
__global__ void __launch_bounds__(32 * FIN_WARPS) k_finalize(FinArgs a)
{
    __shared__ float sM[FIN_WARPS][84];
    __shared__ float sH[FIN_WARPS][144];
    __shared__ float sX[FIN_WARPS][12];
    __shared__ float sS[FIN_WARPS][16];
    __shared__ float sL[FIN_WARPS][144];
    __shared__ int sNk[FIN_WARPS][ED_MAX_KG];
    __shared__ float4 sNg[FIN_WARPS][ED_MAX_KG];
    __shared__ __align__(16) float sNx[FIN_WARPS][12 * ED_MAX_KG];
    // entry table of a 12x12 block: moment index of (R, C) and of (R, 3-column
    // shift), R, C (the same for every block; computed once per CTA)
    __shared__ int s_tab[144];
    ed_pdl_trigger();   // (launched after the join with the pose stream: everything before is complete)
    fill_block_table(s_tab);
    __syncthreads();
    const int wid = threadIdx.x >> 5;
    const int u = blockIdx.x * FIN_WARPS + wid;
    if (u < a.n_upper)
        finalize_block<INV>(a, u, sM[wid], sH[wid], sX[wid], sS[wid], sL[wid], sNk[wid], sNg[wid], sNx[wid], s_tab);
}

// ---------------------------------------------------------------------------
// pose pass (one CTA): pose block and gradient, priors E_r / E_p, the sums
// of the point pass, pose preconditioner
// ---------------------------------------------------------------------------

#define PF_THREADS 1024

#define PF_BATCH 20   // loads in flight per lane (>= 4 * 148 / 32 partials: one round at 640x480)

// sums of the point-pass partials (component k by warp k < 31, lanes striding
// the CTAs, PF_BATCH loads in flight) and of the node energies (all threads,
// then one warp over the warps); s[0..30], ne[0..1]
__device__ __forceinline__ void pf_sums(const float2 *__restrict__ part, int nparts, int pstride,
                                        const float2 *__restrict__ node_energy, int m, double *s, double *ne,
                                        float2 (*wsum)[2])
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (w < 31) {
        const float2 *src = part + (size_t)w * pstride;
        float2 v = make_float2(0.f, 0.f);
        for (int c0 = 0; c0 < nparts; c0 += 32 * PF_BATCH) {
            float2 buf[PF_BATCH];
#pragma unroll
            for (int q = 0; q < PF_BATCH; ++q) {
                const int c = c0 + lane + 32 * q;
                buf[q] = c < nparts ? src[c] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < PF_BATCH; ++q) v = ed_ff_add(v, buf[q]);
        }
        v = ed_ff_warp_sum(v);
        if (lane == 0) s[w] = ed_ff_value(v);
    }
    float2 er = make_float2(0.f, 0.f), eg = er;
    for (int j = t; j < m; j += PF_THREADS) {
        const float2 e = node_energy[j];
        er = ed_ff_add1(er, e.x);
        eg = ed_ff_add1(eg, e.y);
    }
    er = ed_ff_warp_sum(er);
    eg = ed_ff_warp_sum(eg);
    if (lane == 0) {
        wsum[w][0] = er;
        wsum[w][1] = eg;
    }
    __syncthreads();
    if (w == 0) {
        const float2 a = ed_ff_warp_sum(wsum[lane][0]);
        const float2 b = ed_ff_warp_sum(wsum[lane][1]);
        if (lane == 0) {
            ne[0] = ed_ff_value(a);
            ne[1] = ed_ff_value(b);
        }
    }
    __syncthreads();
}

// inverse of the 6x6 pose block Ls (+ jitter tr/6 I; shared memory, one warp,
// one row per lane): Cholesky in place, then forward and back substitution,
// one column per lane, into out[36] (row-major); false on a non-positive pivot
__device__ __forceinline__ bool pose_inverse6(float *Ls, float *rinv, float jitter, float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const float tr = Ls[0] + Ls[7] + Ls[14] + Ls[21] + Ls[28] + Ls[35];
    __syncwarp();
    if (lane < 6) Ls[7 * lane] += jitter * tr / 6.0f;
    __syncwarp();
    bool ok = true;
    for (int c = 0; c < 6; ++c) {
        if (lane == c) {
            float d = Ls[7 * c];
            for (int p = 0; p < c; ++p) d -= Ls[6 * c + p] * Ls[6 * c + p];
            ok = d > 0.f;
            d = sqrtf(fmaxf(d, 1e-30f));
            Ls[7 * c] = d;
            rinv[c] = 1.0f / d;
        }
        __syncwarp();
        if (lane > c && lane < 6) {
            float v = Ls[6 * lane + c];
            for (int p = 0; p < c; ++p) v -= Ls[6 * lane + p] * Ls[6 * c + p];
            Ls[6 * lane + c] = v * rinv[c];
        }
        __syncwarp();
    }
    const bool all_ok = __all_sync(0xffffffffu, ok);
    if (lane < 6) {
        const int col = lane;
        float y[6], xv[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            float v = r == col ? 1.0f : 0.0f;
#pragma unroll
            for (int p = 0; p < r; ++p) v -= Ls[6 * r + p] * y[p];
            y[r] = v * rinv[r];
        }
#pragma unroll
        for (int r = 5; r >= 0; --r) {
            float v = y[r];
#pragma unroll
            for (int p = r + 1; p < 6; ++p) v -= Ls[6 * p + r] * xv[p];
            xv[r] = v * rinv[r];
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) out[6 * r + col] = xv[r];
    }
    return all_ok;
}

__global__ void __launch_bounds__(PF_THREADS) k_pose_part(const float2 *__restrict__ part, int nparts, int pstride,
                                                          const double *__restrict__ pose, ed_solver_params prm,
                                                          float *__restrict__ pose_blk, float *__restrict__ grad,
                                                          double *__restrict__ dmisc, int *__restrict__ status)
{
    __shared__ double s[32];
    __shared__ double ne[2];
    __shared__ double pri[6];
    __shared__ float2 wsum[PF_THREADS / 32][2];
    __shared__ float Ls[36];
    __shared__ float rinv[6];
    const int t = threadIdx.x, lane = t & 31;
    static_assert(PF_BATCH * 32 * 1 >= 4 * 148, "one round of loads on a 148-SM part");
    pf_sums(part, nparts, pstride, nullptr, 0, s, ne, wsum);
    // pose block (+ prior weights on the diagonal, LM damping), one entry per thread;
    // priors and the pose gradient, one coordinate per thread
    if (t < 36) {
        const int a = t / 6, b = t % 6, lo = a < b ? a : b, hi = a < b ? b : a;
        float h = (float)s[2 + 6 * lo - lo * (lo - 1) / 2 + (hi - lo)];
        if (a == b) h = (float)((double)h + (a < 3 ? prm.w_r : prm.w_p)) * (1.0f + prm.lambda);
        pose_blk[t] = h;
        Ls[t] = h;
    } else if (t >= 64 && t < 70) {
        const int a = t - 64;
        const double wt = a < 3 ? prm.w_r : prm.w_p;
        const double d = pose[a] - prm.prior[a];
        pri[a] = wt * d * d;
        grad[a] = (float)(s[23 + a] + wt * d);
    }
    __syncthreads();
    if (t < 32) {
        if (!pose_inverse6(Ls, rinv, prm.jitter, pose_blk + 36) && lane == 0) atomicCAS(status, 0, ED_ERR_BREAKDOWN);
    } else if (t == 32) {
        // for the energy totals k_fin_totals forms after the finalisation (the
        // node energies are not known yet: this pass runs beside the assembly)
        double *ps = dmisc + DM_POSE;
        ps[0] = s[0];
        ps[1] = s[1];
        ps[2] = s[29];
        ps[3] = s[30];
        ps[4] = pri[0] + pri[1] + pri[2];
        ps[5] = pri[3] + pri[4] + pri[5];
    }
}

// ---------------------------------------------------------------------------
// Levenberg-Marquardt acceptance on the device (Sec. II.F solves Eq. 3 with
// LM): the energy at the step's input against that of the last accepted point
// ---------------------------------------------------------------------------

__global__ void k_lm_reset(double *__restrict__ dmisc, int *__restrict__ misc, float lambda0)
{
    dmisc[DM_LAM] = lambda0;
    misc[MI_LM_HAVE] = 0;
    misc[MI_LM_REJECT] = 0;
}

// one thread: reject (restore the accepted point, lambda x 10, 1e-4 from 0) or
// accept (store this point, lambda / 10 after the first); a step whose energy
// is not finite is rejected too when an accepted point exists
__global__ void k_lm_decide(double *__restrict__ dmisc, int *__restrict__ misc, ed_stats *stats)
{
    int rej = 0;
    double lam = dmisc[DM_LAM];
    const int st = misc[MI_STATUS];
    if (st == ED_OK || st == ED_ERR_NONFINITE) {
        const double E = dmisc[0];
        const int have = misc[MI_LM_HAVE];
        if (have && !(E <= dmisc[DM_EPREV])) {
            rej = 1;
            lam = lam > 0.0 ? 10.0 * lam : 1e-4;
            for (int k = 0; k < 8; ++k) dmisc[k] = dmisc[DM_SAVED + k];
            misc[MI_STATUS] = ED_OK;
        } else if (st == ED_OK) {
            if (have) lam *= 0.1;
            dmisc[DM_EPREV] = E;
            for (int k = 0; k < 8; ++k) dmisc[DM_SAVED + k] = dmisc[k];
            misc[MI_LM_HAVE] = 1;
        }
        dmisc[DM_LAM] = lam;
    }
    misc[MI_LM_REJECT] = rej;
    if (stats) {
        if (rej) {
            stats->energy = dmisc[0];
            stats->e_data = dmisc[1];
            stats->e_rot = dmisc[2];
            stats->e_reg = dmisc[3];
            stats->e_rot_prior = dmisc[4];
            stats->e_pos_prior = dmisc[5];
            stats->n_valid = (int)dmisc[6];
            stats->e_corr = dmisc[7];
        }
        stats->lm_rejected = rej;
        stats->lambda = lam;
    }
}

struct LmSwapArgs {
    float4 *bsr, *bsr_s;
    long n_bsr4;
    float4 *pnode, *pnode_s;
    int n_pnode4;
    float4 *x, *x_p;
    int n_x4;
    float *grad, *grad_s;
    int n_grad;
    float *pblk, *pblk_s;   // 36 floats
    double *xm, *xm_p;      // n_xm doubles (0 without the FP64 master)
    int n_xm;
    double *pose, *pose_p;  // 6 doubles
    const int *misc;
};

template <typename T>
__device__ __forceinline__ void lm_move(T *live, T *saved, long n, bool rej, long i0, long stride)
{
    if (rej) {
        for (long k = i0; k < n; k += stride) live[k] = saved[k];
    } else {
        for (long k = i0; k < n; k += stride) saved[k] = live[k];
    }
}

// the undamped system and the parameters: stored on accept, restored on reject
__global__ void __launch_bounds__(512) k_lm_swap(LmSwapArgs a)
{
    if (a.misc[MI_STATUS] != ED_OK) return;
    const bool rej = a.misc[MI_LM_REJECT] != 0;
    const long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x, st = (long)gridDim.x * blockDim.x;
    lm_move(a.bsr, a.bsr_s, a.n_bsr4, rej, i0, st);
    lm_move(a.pnode, a.pnode_s, a.n_pnode4, rej, i0, st);
    lm_move(a.x, a.x_p, a.n_x4, rej, i0, st);
    lm_move(a.grad, a.grad_s, a.n_grad, rej, i0, st);
    lm_move(a.pblk, a.pblk_s, 36, rej, i0, st);
    lm_move(a.xm, a.xm_p, a.n_xm, rej, i0, st);
    lm_move(a.pose, a.pose_p, 6, rej, i0, st);
}

// damping of the diagonal blocks and of the pose block by (1 + lambda) on their
// diagonals, and their block-Jacobi inverses (one warp per node, then the pose)
__global__ void __launch_bounds__(32 * FIN_WARPS) k_lm_precond(const int *__restrict__ diag_pos, int m,
                                                                float *__restrict__ bsr, float *__restrict__ minv,
                                                                float *__restrict__ pose_blk,
                                                                const double *__restrict__ dmisc, float jitter,
                                                                int *__restrict__ misc)
{
    __shared__ float sH[FIN_WARPS][144];
    __shared__ float sL[FIN_WARPS][144];
    __shared__ float sRinv[FIN_WARPS][12];
    if (misc[MI_STATUS] != ED_OK) return;
    const float f = 1.0f + (float)dmisc[DM_LAM];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * FIN_WARPS + wid;
    float *H = sH[wid];
    if (j < m) {
        float *Hb = bsr + (long)diag_pos[j] * 144;
        for (int e = lane; e < 144; e += 32) {
            float h = Hb[e];
            if (e % 13 == 0) {
                h *= f;
                Hb[e] = h;
            }
            H[e] = h;
        }
        __syncwarp();
        if (!block_inverse12(H, sL[wid], jitter, minv + (long)j * 144) && lane == 0)
            atomicCAS(misc + MI_STATUS, 0, ED_ERR_BREAKDOWN);
    } else if (j == m) {
        for (int e = lane; e < 36; e += 32) {
            float h = pose_blk[e];
            if (e % 7 == 0) {
                h *= f;
                pose_blk[e] = h;
            }
            H[e] = h;
        }
        __syncwarp();
        if (!pose_inverse6(H, sRinv[wid], jitter, pose_blk + 36) && lane == 0)
            atomicCAS(misc + MI_STATUS, 0, ED_ERR_BREAKDOWN);
    }
}

static ed_status lm_stage(ed_context *ctx, const ed_solver_params *prm, float *x, double *x_master, double *pose,
                          ed_stats *stats, cudaStream_t st)
{
    const int m = ctx->m;
    k_lm_decide<<<1, 1, 0, st>>>(ctx->dmisc, ctx->misc, stats); ed_note_launch();
    LmSwapArgs la;
    la.bsr = (float4 *)ctx->bsr;
    la.bsr_s = (float4 *)ctx->bsr_s;
    la.n_bsr4 = (long)ctx->nnzb * 36;
    la.pnode = (float4 *)ctx->pnode;
    la.pnode_s = (float4 *)ctx->pnode_s;
    la.n_pnode4 = m * 18;
    la.x = (float4 *)x;
    la.x_p = (float4 *)ctx->x_prev;
    la.n_x4 = m * 3;
    la.grad = ctx->grad;
    la.grad_s = ctx->grad_s;
    la.n_grad = 12 * m + 6;
    la.pblk = ctx->pose_blk;
    la.pblk_s = ctx->pblk_s;
    const bool mixed = prm->precision == ED_PRECISION_MIXED;
    la.xm = mixed ? x_master : nullptr;
    la.xm_p = ctx->xm_prev;
    la.n_xm = mixed ? 12 * m : 0;
    la.pose = pose;
    la.pose_p = ctx->pose_prev;
    la.misc = ctx->misc;
    k_lm_swap<<<2 * ctx->num_sms, 512, 0, st>>>(la); ed_note_launch();
    k_lm_precond<<<ed_div_up(m + 1, FIN_WARPS), 32 * FIN_WARPS, 0, st>>>(ctx->diag_pos, m, ctx->bsr, ctx->minv,
                                                                       ctx->pose_blk, ctx->dmisc, prm->jitter,
                                                                       ctx->misc); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}

extern "C" ed_status ed_lm_reset(ed_context *ctx, float lambda0, cudaStream_t st)
{
    if (!ctx || !(lambda0 >= 0.f) || !isfinite(lambda0)) return ED_ERR_ARG;
    k_lm_reset<<<1, 1, 0, st>>>(ctx->dmisc, ctx->misc, lambda0); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}

static ed_status check_frame(const ed_context *ctx, const ed_frame *fr)
{
    if (!fr || !fr->depth || !fr->nmap || fr->intr.width <= 0 || fr->intr.height <= 0 ||
        fr->intr.width > ctx->lim.max_width || fr->intr.height > ctx->lim.max_height || !(fr->intr.fx > 0.f) ||
        !(fr->intr.fy > 0.f) || ((uintptr_t)fr->nmap & 15))
        return ED_ERR_ARG;
    return ED_OK;
}

// one Gauss-Newton iteration up to the normal equations: association,
// residuals, assembly, block inverses, pose rows
ed_status ed_gn_pre(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, float *x, double *x_master,
                    double *pose, ed_stats *stats, cudaStream_t st, bool fork_pose)
{
    if (!ctx || !prm || !x || !pose || ((uintptr_t)x & 15)) return ED_ERR_ARG;
    if (!ctx->have_graph) return ED_ERR_STATE;
    ed_status s = check_frame(ctx, fr);
    if (s != ED_OK) return s;
    if (prm->n_pcg < 0 || (prm->precision == ED_PRECISION_MIXED && !x_master) ||
        (prm->precision != ED_PRECISION_FP32 && prm->precision != ED_PRECISION_MIXED) ||
        (prm->lm_accept != 0 && prm->lm_accept != 1))
        return ED_ERR_ARG;
    const int m = ctx->m;
    // (the point pass clears the device status word)
    if ((s = ed_point_pass(ctx, fr, prm, x, pose, PASS_STEP, st)) != ED_OK) return s;
    const bool lm = prm->lm_accept != 0;
    // the pose pass (pose block, its inverse, pose gradient, prior energies,
    // the point-pass sums) needs only the point pass: it runs on the context's
    // second stream beside the assembly, joined before the finalisation (in a
    // batch, where other problems fill the GPU, it stays on the step's stream)
    {
        ed_solver_params pf = *prm;
        if (lm) pf.lambda = 0.f;
        cudaStream_t ps = fork_pose ? ctx->aux : st;
        if (fork_pose) {
            ED_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
            ED_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
        }
        k_pose_part<<<1, PF_THREADS, 0, ps>>>(ctx->k1_part, k1_grid(ctx), ctx->max_k1_ctas, pose, pf, ctx->pose_blk,
                                              ctx->grad + 12 * m, ctx->dmisc, ctx->misc + MI_STATUS); ed_note_launch();
        ED_LAUNCH_CHECK();
        if (fork_pose) ED_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->aux));
    }
    if (ctx->n_chunks > 0) {
        const int n0 = ctx->n_chunks0, base1 = ctx->chunk_base1, n1 = ctx->n_chunks - base1;
        ed_tm_begin(ctx, ED_KERNEL_ASSEMBLE, st);
        if (n0 > 0) {
            ED_CUDA_TRY(ed_launch_pdl(k_assemble0, dim3(ed_div_up(2 * n0, 4)), dim3(128), 0, st, (const int4 *)ctx->chunks, n0,
                                      ctx->max_chunks, (const float4 *)ctx->ent_geo, (const uint32_t *)ctx->ent_val,
                                      (const float4 *)ctx->rec0, ctx->partials)); ed_note_launch();
        }
        if (n1 > 0) {
            ED_CUDA_TRY(ed_launch_pdl(k_assemble1, dim3(ed_div_up(2 * n1, 4)), dim3(128), 0, st, (const int4 *)ctx->chunks,
                                      base1, n1, ctx->max_chunks, (const float4 *)ctx->ent_geo,
                                      (const uint32_t *)ctx->ent_val, (const float4 *)ctx->rec0,
                                      (const float4 *)ctx->rec1, (const double *)pose, ctx->partials)); ed_note_launch();
        }
        ed_tm_end(ctx, ED_KERNEL_ASSEMBLE, st);
        ED_LAUNCH_CHECK();
    }
    FinArgs fa;
    fa.info = ctx->fin_info;
    fa.col = ctx->col;
    fa.nbr = ctx->graph.nbr;
    fa.part = ctx->partials;
    fa.max_chunks = ctx->max_chunks;
    fa.n_upper = ctx->n_upper;
    fa.kg = ctx->k_graph;
    fa.mixed = prm->precision == ED_PRECISION_MIXED;
    fa.g = (const float4 *)ctx->graph.nodes;
    fa.x4 = (const float4 *)x;
    fa.w_rot = prm->w_rot;
    fa.w_reg = prm->w_reg;
    fa.lambda = lm ? 0.f : prm->lambda;
    fa.jitter = prm->jitter;
    fa.bsr = ctx->bsr;
    fa.grad = ctx->grad;
    fa.pnode = ctx->pnode;
    fa.minv = ctx->minv;
    fa.node_energy = ctx->node_energy;
    fa.status = ctx->misc + MI_STATUS;
    fa.m = m;
    fa.misc = ctx->misc;
    fa.dmisc = ctx->dmisc;
    fa.stats = stats;
    fa.lambda_report = fa.lambda;
    if (fork_pose) ED_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    ed_tm_begin(ctx, ED_KERNEL_FINALIZE, st);
    (lm ? k_finalize<false> : k_finalize<true>)<<<ed_div_up(ctx->n_upper, FIN_WARPS), 32 * FIN_WARPS, 0, st>>>(fa); ed_note_launch();
    ED_CUDA_TRY(ed_launch_pdl(k_fin_totals, dim3(1), dim3(32 * FIN_WARPS), 0, st, fa)); ed_note_launch();
    ed_tm_end(ctx, ED_KERNEL_FINALIZE, st);
    ED_LAUNCH_CHECK();
    if (lm) return lm_stage(ctx, prm, x, x_master, pose, stats, st);
    return ED_OK;
}

// after the PCG solve (which also applied x += d, pose += d_pose): the
// system of this step can be exported
ed_status ed_gn_post(ed_context *ctx)
{
    ctx->have_system = 1;
    return ED_OK;
}

extern "C" ed_status ed_gn_step(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, float *x,
                                double *x_master, double *pose, ed_stats *stats, cudaStream_t st)
{
    ed_status s = ed_gn_pre(ctx, fr, prm, x, x_master, pose, stats, st);
    if (s != ED_OK) return s;
    if ((s = ed_pcg_solve(ctx, prm, x, x_master, pose, stats, st)) != ED_OK) return s;
    return ed_gn_post(ctx);
}

// blocks (row-major BSR), pose-node blocks, pose block, J^T r, solution
extern "C" ed_status ed_export_system(ed_context *ctx, int *row_ptr, int *col, float *blocks, float *pose_node,
                                      float *pose_block, float *grad, float *delta, cudaStream_t st)
{
    if (!ctx) return ED_ERR_ARG;
    if (!ctx->have_system) return ED_ERR_STATE;
    const int m = ctx->m, P = 12 * m + 6;
    if (row_ptr) ED_CUDA_TRY(cudaMemcpyAsync(row_ptr, ctx->row_ptr, sizeof(int) * (m + 1), cudaMemcpyDeviceToDevice, st));
    if (col) ED_CUDA_TRY(cudaMemcpyAsync(col, ctx->col, sizeof(int) * ctx->nnzb, cudaMemcpyDeviceToDevice, st));
    if (blocks)
        ED_CUDA_TRY(cudaMemcpyAsync(blocks, ctx->bsr, sizeof(float) * 144 * (size_t)ctx->nnzb, cudaMemcpyDeviceToDevice, st));
    if (pose_node)
        ED_CUDA_TRY(cudaMemcpyAsync(pose_node, ctx->pnode, sizeof(float) * 72 * (size_t)m, cudaMemcpyDeviceToDevice, st));
    if (pose_block) ED_CUDA_TRY(cudaMemcpyAsync(pose_block, ctx->pose_blk, sizeof(float) * 36, cudaMemcpyDeviceToDevice, st));
    if (grad) ED_CUDA_TRY(cudaMemcpyAsync(grad, ctx->grad, sizeof(float) * P, cudaMemcpyDeviceToDevice, st));
    if (delta) ED_CUDA_TRY(cudaMemcpyAsync(delta, ctx->vec, sizeof(float) * P, cudaMemcpyDeviceToDevice, st));
    return ED_OK;
}

// ---------------------------------------------------------------------------
// energy of Eq. (3) and its gradient (differentiation of the warp + energy)
// ---------------------------------------------------------------------------

// rot and reg energies per node (no normal equations)
__global__ void k_node_energy(int m, int kg, const int *__restrict__ nbr, const float4 *__restrict__ g,
                              const float4 *__restrict__ x4, float w_rot, float w_reg, float2 *__restrict__ ne)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const float *X = &x4[3 * j].x;
    float er = 0.f, eg = 0.f;
    const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {1, 2, 2, 0, 1, 2};
    for (int q = 0; q < 6; ++q) {
        float rho = X[pa[q]] * X[pb[q]] + X[4 + pa[q]] * X[4 + pb[q]] + X[8 + pa[q]] * X[8 + pb[q]];
        if (pa[q] == pb[q]) rho -= 1.0f;
        er += w_rot * rho * rho;
    }
    const float4 gj = g[j];
    for (int s = 0; s < kg; ++s) {
        const int k = nbr[j * kg + s];
        if (k < 0) continue;
        const float4 gk = g[k];
        const float hh[3] = {gk.x - gj.x, gk.y - gj.y, gk.z - gj.z};
        const float *xk = &x4[3 * k].x;
        for (int r = 0; r < 3; ++r) {
            const float e = ed_reg_residual(X + 4 * r, r, hh, xk[4 * r + 3]);
            eg += w_reg * e * e;
        }
    }
    ne[j] = make_float2(er, eg);
}

__global__ void __launch_bounds__(PF_THREADS) k_energy_final(const float2 *__restrict__ part, int nparts, int pstride,
                                                              const float2 *__restrict__ node_energy, int m,
                                                              const double *__restrict__ pose, ed_solver_params prm,
                                                              int has_corr, double *__restrict__ out)
{
    __shared__ double s[32];
    __shared__ double ne[2];
    __shared__ float2 wsum[PF_THREADS / 32][2];
    pf_sums(part, nparts, pstride, node_energy, m, s, ne, wsum);
    if (threadIdx.x == 0) {
        double Er = 0.0, Ep = 0.0;
        for (int q = 0; q < 6; ++q) {
            const double d = pose[q] - prm.prior[q];
            if (q < 3) Er += prm.w_r * d * d;
            else Ep += prm.w_p * d * d;
        }
        out[0] = s[0] + ne[0] + ne[1] + Er + Ep + s[30];
        out[1] = s[0];
        out[2] = ne[0];
        out[3] = ne[1];
        out[4] = Er;
        out[5] = Ep;
        if (has_corr) out[6] = s[30];
    }
}

extern "C" ed_status ed_energy(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, const float *x,
                               const double *pose, double *energy_out, cudaStream_t st)
{
    if (!ctx || !prm || !x || !pose || !energy_out || ((uintptr_t)x & 15)) return ED_ERR_ARG;
    if (!ctx->have_graph) return ED_ERR_STATE;
    ed_status s = check_frame(ctx, fr);
    if (s != ED_OK) return s;
    if ((s = ed_point_pass(ctx, fr, prm, x, pose, PASS_ENERGY, st)) != ED_OK) return s;
    k_node_energy<<<ed_div_up(ctx->m, 128), 128, 0, st>>>(ctx->m, ctx->k_graph, ctx->graph.nbr,
                                                          (const float4 *)ctx->graph.nodes, (const float4 *)x,
                                                          prm->w_rot, prm->w_reg, ctx->node_energy); ed_note_launch();
    k_energy_final<<<1, PF_THREADS, 0, st>>>(ctx->k1_part, k1_grid(ctx), ctx->max_k1_ctas, ctx->node_energy, ctx->m,
                                              pose, *prm, ctx->n_kp > 0, energy_out); ed_note_launch();
    ED_LAUNCH_CHECK();
    ctx->have_energy = 1;
    return ED_OK;
}

// dE/dx_j = 2 [ sum_i r_i w_ij sqrt(w) (R^T n) (x) d^_ij  +  rot and reg terms ]
// (Gaussian w_ij recomputed from the node indices, not read from the graph),
// gathered per node over the points of its diagonal block (fixed order)
__global__ void __launch_bounds__(128) k_grad_nodes(int m, int kg, const int *__restrict__ nbr,
                                                    const int *__restrict__ row_ptr, const int *__restrict__ col,
                                                    const int *__restrict__ diag_pos, const int *__restrict__ ent_start,
                                                    const int *__restrict__ ent_cnt, const uint32_t *__restrict__ ent,
                                                    const float4 *__restrict__ g, const float4 *__restrict__ x4,
                                                    const float4 *__restrict__ pos, const float *__restrict__ wts,
                                                    const ushort4 *__restrict__ idx, int recompute_w, float sigma,
                                                    const float4 *__restrict__ gp0, float w_rot, float w_reg,
                                                    float scale, float *__restrict__ grad)
{
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 4 + wid;
    if (j >= m) return;
    const int b = diag_pos[j];
    const int e0 = ent_start[b], ne = ent_cnt[b];
    const float4 gj = g[j];
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.f;
    for (int e = e0 + lane; e < e0 + ne; e += 32) {
        const uint32_t v = ent[e];
        const int i = (int)(v >> 4), s = (v >> 2) & 3;
        const float4 r0 = gp0[i];
        const float4 p = pos[i];
        float ws;
        if (recompute_w) {
            const float4 w4 = ed_gauss_weights(p, idx[i], g, m, sigma);
            ws = s == 0 ? w4.x : s == 1 ? w4.y : s == 2 ? w4.z : w4.w;
        } else {
            ws = wts[4 * i + s];
        }
        const float c = ws * r0.w;
        const float dh[4] = {p.x - gj.x, p.y - gj.y, p.z - gj.z, 1.0f};
        const float nb[3] = {r0.x, r0.y, r0.z};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[4 * r + k] += c * nb[r] * dh[k];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane != 0) return;
    const float *X = &x4[3 * j].x;
    // Rot(A_j): d rho / d A[r][a] (columns a, b)
    const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {1, 2, 2, 0, 1, 2};
    for (int q = 0; q < 6; ++q) {
        const int ca = pa[q], cb = pb[q];
        float rho = X[ca] * X[cb] + X[4 + ca] * X[4 + cb] + X[8 + ca] * X[8 + cb];
        if (ca == cb) rho -= 1.0f;
        for (int r = 0; r < 3; ++r) {
            acc[4 * r + ca] += w_rot * rho * X[4 * r + cb];
            acc[4 * r + cb] += w_rot * rho * X[4 * r + ca];
        }
    }
    for (int s = 0; s < kg; ++s) {             // out-edges j -> k
        const int k = nbr[j * kg + s];
        if (k < 0) continue;
        const float4 gk = g[k];
        const float hh[4] = {gk.x - gj.x, gk.y - gj.y, gk.z - gj.z, 1.0f};
        const float *xk = &x4[3 * k].x;
        for (int r = 0; r < 3; ++r) {
            const float e = ed_reg_residual(X + 4 * r, r, hh, xk[4 * r + 3]);
            for (int c = 0; c < 4; ++c) acc[4 * r + c] += w_reg * e * hh[c];
        }
    }
    for (int t = row_ptr[j]; t < row_ptr[j + 1]; ++t) {   // in-edges k -> j lie in row j
        const int k = col[t];
        bool in = false;
        for (int s = 0; s < kg; ++s) in |= nbr[k * kg + s] == j;
        if (!in || k == j) continue;
        const float4 gk = g[k];
        const float hh[3] = {gj.x - gk.x, gj.y - gk.y, gj.z - gk.z};
        const float *xk = &x4[3 * k].x;
        for (int r = 0; r < 3; ++r) {
            const float e = ed_reg_residual(xk + 4 * r, r, hh, X[4 * r + 3]);
            acc[4 * r + 3] -= w_reg * e;
        }
    }
    for (int k = 0; k < 12; ++k) grad[12 * j + k] = 2.0f * scale * acc[k];
}

__global__ void k_grad_pose(const float2 *__restrict__ part, int nparts, int pstride, const double *__restrict__ pose,
                            ed_solver_params prm, float scale, float *__restrict__ gpose)
{
    const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;   // warp t: pose coordinate t
    if (t >= 6) return;
    const float2 *src = part + (size_t)(23 + t) * pstride;
    float2 v = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int c = lane; c < nparts; c += 32) v = ed_ff_add(v, src[c]);
    v = ed_ff_warp_sum(v);
    if (lane == 0) {
        const double w = t < 3 ? prm.w_r : prm.w_p;
        gpose[t] = (float)(2.0 * scale * (ed_ff_value(v) + w * (pose[t] - prm.prior[t])));
    }
}

extern "C" ed_status ed_energy_grad(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, const float *x,
                                    const double *pose, float grad_scale, float *grad_x, float *grad_pose,
                                    cudaStream_t st)
{
    if (!ctx || !prm || !x || !pose || !grad_x || !grad_pose || ((uintptr_t)x & 15)) return ED_ERR_ARG;
    if (!ctx->have_graph || !ctx->have_energy) return ED_ERR_STATE;
    ed_status s = check_frame(ctx, fr);
    if (s != ED_OK) return s;
    if ((s = ed_point_pass(ctx, fr, prm, x, pose, PASS_GRAD, st)) != ED_OK) return s;
    k_grad_nodes<<<ed_div_up(ctx->m, 4), 128, 0, st>>>(ctx->m, ctx->k_graph, ctx->graph.nbr, ctx->row_ptr, ctx->col,
                                                       ctx->diag_pos,
                                                       ctx->ent_start, ctx->ent_cnt, ctx->ent_val,
                                                       (const float4 *)ctx->graph.nodes, (const float4 *)x,
                                                       (const float4 *)ctx->pos, ctx->graph.weights,
                                                       (const ushort4 *)ctx->graph.idx,
                                                       ctx->weight_mode == ED_WEIGHT_GAUSSIAN, ctx->sigma, ctx->gpts,
                                                       prm->w_rot, prm->w_reg, grad_scale, grad_x); ed_note_launch();
    k_grad_pose<<<1, 192, 0, st>>>(ctx->k1_part, k1_grid(ctx), ctx->max_k1_ctas, pose, *prm, grad_scale, grad_pose); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}
