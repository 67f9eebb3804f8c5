// maintain.cu -- model maintenance across frames: box downsampling of the
// point model (Sec. III.A; Algorithm 3, first line) and the back-projection
// error of a warped model against a depth image (Sec. III).
#include <math.h>

#include "ed_internal.cuh"

// ---------------------------------------------------------------------------
// box downsampling
// ---------------------------------------------------------------------------

// box grid anchored at the bounding-box minimum: boxes per axis
// floor((max - min) / box) + 1 by the FP32 rule of the keys below
__global__ void k_vox_setup(int *misc, float *fmisc, float box)
{
    long cells = 1;
    for (int d = 0; d < 3; ++d) {
        const float mn = o2f(misc[MI_BBOX + d]), mx = o2f(misc[MI_BBOX + 3 + d]);
        const int n = (int)floorf(__fdiv_rn(__fsub_rn(mx, mn), box)) + 1;
        misc[MI_VOX + d] = n;
        fmisc[MF_VOX + d] = mn;
        cells *= n;
    }
    misc[MI_VOX + 3] = cells < 4294967296L ? ED_OK : ED_ERR_CAPACITY;
}

// key of every point: ix + nx (iy + ny iz), ix = floor((x - min) / box) in FP32
__global__ void k_vox_key(const float4 *__restrict__ pos, int n, const int *__restrict__ misc,
                          const float *__restrict__ fmisc, float box, uint32_t *__restrict__ key,
                          uint32_t *__restrict__ val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos[i];
    const float c[3] = {p.x, p.y, p.z};
    uint32_t k = 0, stride = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int nd = misc[MI_VOX + d];
        int b = (int)floorf(__fdiv_rn(__fsub_rn(c[d], fmisc[MF_VOX + d]), box));
        b = min(max(b, 0), nd - 1);
        k += (uint32_t)b * stride;
        stride *= (uint32_t)nd;
    }
    key[i] = k;
    val[i] = (uint32_t)i;
}

__global__ void k_vox_start(const uint32_t *__restrict__ key, int n, int *__restrict__ start)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    start[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// one thread per box (at the box's first sorted point): the box's points in
// increasing index order, omega-weighted means of position, colour and normal
// (normalised), capped weight sum, latest time stamp, stability flag
__global__ void k_vox_merge(const uint32_t *__restrict__ key, const uint32_t *__restrict__ idx,
                            const int *__restrict__ start, const int *__restrict__ slot, int n,
                            const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                            const float4 *__restrict__ col, const int *__restrict__ tstamp, ed_downsample_params P,
                            int capacity, float4 *__restrict__ pos_out, float4 *__restrict__ nrm_out,
                            float4 *__restrict__ col_out, int *__restrict__ t_out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n || !start[a]) return;
    const int o = slot[a];
    if (o >= capacity) return;
    const uint32_t k = key[a];
    float sw = 0.f, cw = 0.f;
    float sp[3] = {0.f, 0.f, 0.f}, sn[3] = {0.f, 0.f, 0.f}, sc[4] = {0.f, 0.f, 0.f, 0.f};
    float up[3] = {0.f, 0.f, 0.f}, un[3] = {0.f, 0.f, 0.f}, uc[4] = {0.f, 0.f, 0.f, 0.f};
    int tmax = tstamp[idx[a]];
    for (int j = a; j < n && key[j] == k; ++j) {
        const int i = (int)idx[j];
        const float4 p = pos[i], nn = nrm[i], c = col[i];
        const float w = p.w;
        sw += w;
        cw += 1.f;
        sp[0] += w * p.x; sp[1] += w * p.y; sp[2] += w * p.z;
        sn[0] += w * nn.x; sn[1] += w * nn.y; sn[2] += w * nn.z;
        sc[0] += w * c.x; sc[1] += w * c.y; sc[2] += w * c.z; sc[3] += w * c.w;
        up[0] += p.x; up[1] += p.y; up[2] += p.z;
        un[0] += nn.x; un[1] += nn.y; un[2] += nn.z;
        uc[0] += c.x; uc[1] += c.y; uc[2] += c.z; uc[3] += c.w;
        tmax = max(tmax, tstamp[i]);
    }
    const float w_out = fminf(sw, P.omega_max);
    if (!(sw > 0.f)) {   // no weight in the box: a plain average
        sw = cw;
        for (int d = 0; d < 3; ++d) { sp[d] = up[d]; sn[d] = un[d]; }
        for (int d = 0; d < 4; ++d) sc[d] = uc[d];
    }
    const float l2 = sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2];
    const float il = l2 > 0.f ? rsqrtf(l2) : 0.f;
    pos_out[o] = make_float4(sp[0] / sw, sp[1] / sw, sp[2] / sw, w_out);
    nrm_out[o] = make_float4(sn[0] * il, sn[1] * il, sn[2] * il, w_out >= P.tau_weight ? 1.0f : 0.0f);
    col_out[o] = make_float4(sc[0] / sw, sc[1] / sw, sc[2] / sw, sc[3] / sw);
    t_out[o] = tmax;
}

__global__ void k_vox_count(const int *__restrict__ total, int capacity, int *__restrict__ out)
{
    const int tot = *total;
    out[0] = tot < capacity ? tot : capacity;
    out[1] = tot > capacity ? ED_ERR_CAPACITY : ED_OK;
}

extern "C" ed_status ed_downsample(ed_context *ctx, const float *pos, const float *nrm, const float *col,
                                   const int *tstamp, int n_in, const ed_downsample_params *P, int capacity,
                                   float *pos_out, float *nrm_out, float *col_out, int *t_out, int *counts_out,
                                   cudaStream_t st)
{
    if (!ctx || !P || !counts_out || n_in < 0 || n_in > ctx->lim.max_points || capacity < 0 || !(P->box > 0.f) ||
        !isfinite(P->box))
        return ED_ERR_ARG;
    if (n_in == 0) {   // nothing to merge (the arrays may be NULL)
        ED_CUDA_TRY(cudaMemsetAsync(counts_out, 0, 2 * sizeof(int), st));
        return ED_OK;
    }
    if (!pos || !nrm || !col || !tstamp || !pos_out || !nrm_out || !col_out || !t_out) return ED_ERR_ARG;
    if (((uintptr_t)pos & 15) || ((uintptr_t)nrm & 15) || ((uintptr_t)col & 15) || ((uintptr_t)pos_out & 15) ||
        ((uintptr_t)nrm_out & 15) || ((uintptr_t)col_out & 15))
        return ED_ERR_ARG;
    if (pos == pos_out || nrm == nrm_out || col == col_out || (const float *)tstamp == (const float *)t_out)
        return ED_ERR_ARG;
    const float4 *P4 = (const float4 *)pos;
    ed_status s;
    if ((s = ed_bbox_enqueue(ctx, P4, n_in, st)) != ED_OK) return s;
    k_vox_setup<<<1, 1, 0, st>>>(ctx->misc, ctx->fmisc, P->box); ed_note_launch();
    ED_LAUNCH_CHECK();
    // the key width of the sort: one read of the grid dims
    int hd[4];
    ED_CUDA_TRY(cudaMemcpyAsync(hd, ctx->misc + MI_VOX, sizeof(hd), cudaMemcpyDeviceToHost, st));
    ED_CUDA_TRY(cudaStreamSynchronize(st));
    if (hd[3] != ED_OK) return ED_ERR_CAPACITY;
    const unsigned long long cells = (unsigned long long)hd[0] * hd[1] * hd[2];
    int bits = 1;
    while (bits < 32 && (1ull << bits) < cells) ++bits;
    k_vox_key<<<ed_div_up(n_in, 256), 256, 0, st>>>(P4, n_in, ctx->misc, ctx->fmisc, P->box, ctx->ent_key,
                                                   ctx->ent_val); ed_note_launch();
    ED_LAUNCH_CHECK();
    if ((s = ed_radix_sort_pairs(ctx, ctx->ent_key, ctx->ent_val, n_in, bits, st)) != ED_OK) return s;
    k_vox_start<<<ed_div_up(n_in, 256), 256, 0, st>>>(ctx->ent_key, n_in, ctx->flag_a); ed_note_launch();
    ED_LAUNCH_CHECK();
    if ((s = ed_scan_exclusive(ctx, ctx->flag_a, ctx->flag_b, n_in, st)) != ED_OK) return s;
    k_vox_merge<<<ed_div_up(n_in, 256), 256, 0, st>>>(ctx->ent_key, ctx->ent_val, ctx->flag_a, ctx->flag_b, n_in, P4,
                                                     (const float4 *)nrm, (const float4 *)col, tstamp, *P, capacity,
                                                     (float4 *)pos_out, (float4 *)nrm_out, (float4 *)col_out,
                                                     t_out); ed_note_launch();
    k_vox_count<<<1, 1, 0, st>>>(ctx->flag_b + n_in, capacity, counts_out); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}

// ---------------------------------------------------------------------------
// back-projection error
// ---------------------------------------------------------------------------

__global__ void k_de_zbuf(const float4 *__restrict__ wpos, int n, ed_intrinsics K, unsigned long long *__restrict__ zb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = wpos[i];
    int u, v;
    if (!ed_project(p.x, p.y, p.z, K, u, v)) return;
    atomicMin(zb + (v * K.width + u), ((unsigned long long)__float_as_uint(p.z) << 32) | (unsigned)i);
}

#define DE_T 256

// per CTA (grid-stride over pixels): sum |z - D|, count, max |z - D|, sum (z - D)^2
__global__ void __launch_bounds__(DE_T) k_de_pixels(const unsigned long long *__restrict__ zb,
                                                    const float4 *__restrict__ wpos, const float *__restrict__ depth,
                                                    int npx, double *__restrict__ part)
{
    __shared__ double sh[4][DE_T / 32];
    double a = 0.0, c = 0.0, mx = 0.0, s2 = 0.0;
    for (int q = blockIdx.x * DE_T + threadIdx.x; q < npx; q += gridDim.x * DE_T) {
        const unsigned long long key = zb[q];
        const float D = depth[q];
        if (key == ~0ull || !(D > 0.f)) continue;
        const double e = (double)wpos[key & 0xffffffffu].z - (double)D;
        a += fabs(e);
        c += 1.0;
        mx = fmax(mx, fabs(e));
        s2 += e * e;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = c;
        sh[2][w] = mx;
        sh[3][w] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double r = 0.0;
        for (int k = 0; k < DE_T / 32; ++k) r = threadIdx.x == 2 ? fmax(r, sh[2][k]) : r + sh[threadIdx.x][k];
        part[(size_t)threadIdx.x * ED_MAX_PCG_GRID + blockIdx.x] = r;
    }
}

// the CTA partials in CTA order
__global__ void k_de_final(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    if (threadIdx.x < 4) {
        double r = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double v = part[(size_t)threadIdx.x * ED_MAX_PCG_GRID + b];
            r = threadIdx.x == 2 ? fmax(r, v) : r + v;
        }
        out[threadIdx.x] = r;
    }
}

extern "C" ed_status ed_depth_error(ed_context *ctx, const float *wpos, int n_points, const float *depth,
                                    ed_intrinsics intr, double *out, cudaStream_t st)
{
    if (!ctx || (!wpos && n_points > 0) || !depth || !out || n_points < 0 || n_points > ctx->lim.max_points || intr.width <= 0 ||
        intr.height <= 0 || intr.width > ctx->lim.max_width || intr.height > ctx->lim.max_height ||
        !(intr.fx > 0.f) || !(intr.fy > 0.f) || ((uintptr_t)wpos & 15))
        return ED_ERR_ARG;
    const int npx = intr.width * intr.height;
    ED_CUDA_TRY(cudaMemsetAsync(ctx->zbuf, 0xff, sizeof(unsigned long long) * npx, st));
    if (n_points > 0) {
        k_de_zbuf<<<ed_div_up(n_points, 256), 256, 0, st>>>((const float4 *)wpos, n_points, intr, ctx->zbuf); ed_note_launch();
    }
    const int nb = min(ed_div_up(npx, DE_T), 2 * ctx->num_sms);
    k_de_pixels<<<nb, DE_T, 0, st>>>(ctx->zbuf, (const float4 *)wpos, depth, npx, ctx->red_part); ed_note_launch();
    k_de_final<<<1, 32, 0, st>>>(ctx->red_part, nb, out); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}
