// fuse.cu -- ed_fuse: model update with a new observation (Sec. II.G,
// Algorithms 1-3, Eqs. fusion1-4), out of place.
#include "ed_internal.cuh"

// Reg, step 1: z-buffer of the warped points, key = (z bits, point index)
// the z-buffer and the fused-pixel marks of the old points cleared to all
// ones (empty pixel, no pixel)
__global__ void k_fuse_init(unsigned long long *__restrict__ zb, int npx, int *__restrict__ fused_pix, int n)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npx) zb[i] = ~0ull;
    if (i < n) fused_pix[i] = -1;
}

__global__ void k_fuse_zbuf(const float4 *__restrict__ wpos, int n, ed_intrinsics K, unsigned long long *__restrict__ zb)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = wpos[i];
    int u, v;
    if (!ed_project(p.x, p.y, p.z, K, u, v)) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(p.z) << 32) | (unsigned)i;
    atomicMin(zb + (v * K.width + u), key);
}

// Algorithm 1 on every pixel of Reg; marks registered points and the pixels to lift
__global__ void k_fuse_reg(const unsigned long long *__restrict__ zb, const float4 *__restrict__ wpos,
                           const float4 *__restrict__ wnrm, const float *__restrict__ depth,
                           const float4 *__restrict__ nmap, int npx, float tau_d, float cos_delta,
                           int *__restrict__ reg, int *__restrict__ fused_pix, int *__restrict__ lift)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npx) return;
    const unsigned long long key = zb[q];
    const float D = depth[q];
    const float4 tn = nmap[q];
    const bool obs = D > 0.f && tn.w != 0.f;
    int r = -1;
    if (key != ~0ull && obs) {
        const int i = (int)(key & 0xffffffffu);
        const float4 p = wpos[i], nn = wnrm[i];
        if (fabsf(__fsub_rn(p.z, D)) < tau_d && ed_dot3_exact(nn.x, nn.y, nn.z, tn.x, tn.y, tn.z) > cos_delta) {
            r = i;
            fused_pix[i] = q;
        }
    }
    reg[q] = r;
    lift[q] = (r < 0 && obs) ? 1 : 0;
}

__global__ void k_fuse_keep(const float4 *__restrict__ pos, const int *__restrict__ tstamp,
                            const int *__restrict__ fused_pix, int n, int frame, int tau_time, float tau_weight,
                            int *__restrict__ keep)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool del = fused_pix[i] < 0 && (frame - tstamp[i]) > tau_time && pos[i].w < tau_weight;
    keep[i] = del ? 0 : 1;
}

__global__ void k_fuse_write_old(const float4 *__restrict__ pos, const float4 *__restrict__ col,
                                 const int *__restrict__ tstamp, const float4 *__restrict__ wpos,
                                 const float4 *__restrict__ wnrm, const int *__restrict__ fused_pix,
                                 const int *__restrict__ keep_scan, int n, const float *__restrict__ depth,
                                 const float4 *__restrict__ nmap, const float4 *__restrict__ color, ed_fuse_params F,
                                 int capacity, float4 *__restrict__ pos_out, float4 *__restrict__ nrm_out,
                                 float4 *__restrict__ col_out, int *__restrict__ t_out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = keep_scan[i];
    if (keep_scan[i + 1] == o || o >= capacity) return;
    float4 p = wpos[i], nn = wnrm[i], c = col[i];
    float w = pos[i].w;
    int t = tstamp[i];
    const int q = fused_pix[i];
    if (q >= 0) {
        // Eqs. fusion1-4 with observation weight 1
        const float D = depth[q];
        const float z = p.z;
        const float Df = (z * w + D) / (w + 1.0f);
        const float s = Df / z;
        p.x *= s;
        p.y *= s;
        p.z *= s;
        const float4 tn = nmap[q], tc = color[q];
        float nx = nn.x * w + tn.x, ny = nn.y * w + tn.y, nz = nn.z * w + tn.z;
        const float l2 = nx * nx + ny * ny + nz * nz;
        const float il = l2 > 0.f ? rsqrtf(l2) : 0.f;
        nn.x = nx * il;
        nn.y = ny * il;
        nn.z = nz * il;
        const float iw = 1.0f / (w + 1.0f);
        c = make_float4((c.x * w + tc.x) * iw, (c.y * w + tc.y) * iw, (c.z * w + tc.z) * iw, (c.w * w + tc.w) * iw);
        w = fminf(w + 1.0f, F.omega_max);
        t = F.frame;
    }
    pos_out[o] = make_float4(p.x, p.y, p.z, w);
    nrm_out[o] = make_float4(nn.x, nn.y, nn.z, w >= F.tau_weight ? 1.0f : 0.0f);
    col_out[o] = c;
    t_out[o] = t;
}

__global__ void k_fuse_write_new(const int *__restrict__ lift_scan, int npx, const int *__restrict__ kept_total,
                                 const float *__restrict__ depth, const float4 *__restrict__ nmap,
                                 const float4 *__restrict__ color, ed_intrinsics K, ed_fuse_params F, int capacity,
                                 float4 *__restrict__ pos_out, float4 *__restrict__ nrm_out, float4 *__restrict__ col_out,
                                 int *__restrict__ t_out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npx) return;
    if (lift_scan[q + 1] == lift_scan[q]) return;
    const int o = *kept_total + lift_scan[q];
    if (o >= capacity) return;
    const int u = q % K.width, v = q / K.width;
    const float D = depth[q];
    const float4 tn = nmap[q];
    pos_out[o] = make_float4(((float)u - K.cx) * D / K.fx, ((float)v - K.cy) * D / K.fy, D, 1.0f);
    nrm_out[o] = make_float4(tn.x, tn.y, tn.z, 1.0f >= F.tau_weight ? 1.0f : 0.0f);
    col_out[o] = color[q];
    t_out[o] = F.frame;
}

__global__ void k_fuse_count(const int *__restrict__ kept_total, const int *__restrict__ lift_total, int capacity,
                             int *__restrict__ out)
{
    ed_pdl_wait();
    ed_pdl_trigger();
    const long tot = (long)*kept_total + *lift_total;
    out[0] = (int)(tot < capacity ? tot : capacity);
    out[1] = tot > capacity ? ED_ERR_CAPACITY : ED_OK;
}

extern "C" ed_status ed_fuse(ed_context *ctx, const float *pos, const float *nrm, const float *col, const int *tstamp,
                             int n_in, const float *wpos, const float *wnrm, const ed_frame *fr,
                             const ed_fuse_params *F, int capacity, float *pos_out, float *nrm_out, float *col_out,
                             int *t_out, int *counts_out, int *reg_out, cudaStream_t st)
{
    (void)nrm;
    if (!ctx || !fr || !F || !pos_out || !nrm_out || !col_out || !t_out || !counts_out || n_in < 0 || capacity < 0 ||
        n_in > ctx->lim.max_points)
        return ED_ERR_ARG;
    if (n_in > 0 && (!pos || !col || !tstamp || !wpos || !wnrm)) return ED_ERR_ARG;   // (NULL allowed for no model)
    if (!fr->depth || !fr->nmap || !fr->color || fr->intr.width <= 0 || fr->intr.height <= 0 ||
        fr->intr.width > ctx->lim.max_width || fr->intr.height > ctx->lim.max_height)
        return ED_ERR_ARG;
    const int npx = fr->intr.width * fr->intr.height;
    int *reg = reg_out ? reg_out : ctx->regpix;
    int *keep = ctx->flag_a, *lift = ctx->flag_b;
    ED_LAUNCH(k_fuse_init, ed_div_up(npx > n_in ? npx : n_in, 256), 256, st, ctx->zbuf, npx, ctx->fused_pix, n_in);
    ed_note_launch();
    if (n_in > 0) {
        ED_LAUNCH(k_fuse_zbuf, ed_div_up(n_in, 256), 256, st, (const float4 *)wpos, n_in, fr->intr, ctx->zbuf); ed_note_launch();
        ED_LAUNCH_CHECK();
    }
    ED_LAUNCH(k_fuse_reg, ed_div_up(npx, 256), 256, st, ctx->zbuf, (const float4 *)wpos, (const float4 *)wnrm, fr->depth,
                                                    (const float4 *)fr->nmap, npx, F->tau_d, F->cos_delta, reg,
                                                    ctx->fused_pix, lift); ed_note_launch();
    ED_LAUNCH_CHECK();
    ed_status s;
    if (n_in > 0) {
        ED_LAUNCH(k_fuse_keep, ed_div_up(n_in, 256), 256, st, (const float4 *)pos, tstamp, ctx->fused_pix, n_in, F->frame,
                                                          F->tau_time, F->tau_weight, keep); ed_note_launch();
        ED_LAUNCH_CHECK();
    }
    if ((s = ed_scan_exclusive(ctx, keep, keep, n_in, st)) != ED_OK) return s;
    if ((s = ed_scan_exclusive(ctx, lift, lift, npx, st)) != ED_OK) return s;
    if (n_in > 0) {
        ED_LAUNCH(k_fuse_write_old, ed_div_up(n_in, 256), 256, st, 
            (const float4 *)pos, (const float4 *)col, tstamp, (const float4 *)wpos, (const float4 *)wnrm, ctx->fused_pix,
            keep, n_in, fr->depth, (const float4 *)fr->nmap, (const float4 *)fr->color, *F, capacity, (float4 *)pos_out,
            (float4 *)nrm_out, (float4 *)col_out, t_out); ed_note_launch();
        ED_LAUNCH_CHECK();
    }
    ED_LAUNCH(k_fuse_write_new, ed_div_up(npx, 256), 256, st, lift, npx, keep + n_in, fr->depth, (const float4 *)fr->nmap,
                                                          (const float4 *)fr->color, fr->intr, *F, capacity,
                                                          (float4 *)pos_out, (float4 *)nrm_out, (float4 *)col_out, t_out); ed_note_launch();
    ED_LAUNCH(k_fuse_count, 1, 1, st, keep + n_in, lift + npx, capacity, counts_out); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}
