// noalloc.cu -- the Eq. (3) energy for callers that cannot allocate device
// memory.
//
// Some callers of this library cannot call cudaMalloc at all: code running
// inside a host framework that owns every device allocation (a plugin that
// may only touch the buffers it is handed), or a real-time loop that forbids
// allocation after start up.  ed_energy_noalloc serves them: it needs no
// context and no workspace.
// Its only scratch -- the per-CTA partial sums of the reduction -- lives in a
// fixed-size array in device global memory, defined at file scope below.
// Every GPU that loads the library holds that array until the process exits.
#include <mutex>

#include "ed_internal.cuh"

#define NA_THREADS 256
#define NA_MAX_POINT_CTAS 8192   // at most 8192 * 256 = 2,097,152 points per call
#define NA_MAX_NODE_CTAS 128     // at most 128 * 256 = 32,768 nodes per call
#define NA_MAX_POINTS (NA_MAX_POINT_CTAS * NA_THREADS)
#define NA_MAX_NODES (NA_MAX_NODE_CTAS * NA_THREADS)

// 2 doubles per point CTA (data energy, valid count) and per node CTA (rot,
// reg energy): 133,120 bytes.  Every call writes every slot it later reads, so
// nothing has to be cleared; calls that overlap on the GPU share the array
// and race.
static __device__ __align__(256) double g_na_scratch[2 * NA_MAX_POINT_CTAS + 2 * NA_MAX_NODE_CTAS];

struct NaPointArgs {
    const float4 *pos, *nrm, *w, *g, *x4;
    const ushort4 *idx;
    const double *pose;
    const float *depth;
    const float4 *nmap;
    ed_intrinsics K;
    int n;
    float eps2, cos_eps_n, sw;
    double *part;
};

__device__ __forceinline__ double na_block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < NA_THREADS / 32; ++k) s += sh[k];
    __syncthreads();
    return s;   // valid in thread 0
}

// one point per thread: Eq. (1) warp, visible-point gate, squared data residual
__global__ void __launch_bounds__(NA_THREADS) k_na_points(NaPointArgs a)
{
    __shared__ ed_pose_f P;
    __shared__ double sh[NA_THREADS / 32];
    if (threadIdx.x == 0) ed_pose_eval(a.pose, P);
    __syncthreads();
    const int i = blockIdx.x * NA_THREADS + threadIdx.x;
    double e = 0.0, c = 0.0;
    if (i < a.n) {
        const ed_warped W = ed_warp_point(a.pos[i], a.nrm[i], a.idx[i], a.w[i], a.g, a.x4, P.R, P.T);
        const int q = ed_associate(W, a.depth, a.nmap, a.K, a.eps2, a.cos_eps_n);
        if (q >= 0) {
            const int u = q % a.K.width, v = q / a.K.width;
            const float D = __ldg(a.depth + q);
            const float4 tn = __ldg(a.nmap + q);
            const float Gx = ((float)u - a.K.cx) * D / a.K.fx, Gy = ((float)v - a.K.cy) * D / a.K.fy;
            const float r = a.sw * (tn.x * (W.v.x - Gx) + tn.y * (W.v.y - Gy) + tn.z * (W.v.z - D));
            e = (double)r * (double)r;
            c = 1.0;
        }
    }
    const double se = na_block_sum(e, sh);
    const double sc = na_block_sum(c, sh);
    if (threadIdx.x == 0) {
        a.part[2 * blockIdx.x] = se;
        a.part[2 * blockIdx.x + 1] = sc;
    }
}

// one node per thread: Rot(A_j) and the E_reg residuals of the edges leaving j
__global__ void __launch_bounds__(NA_THREADS) k_na_nodes(int m, int kg, const int *__restrict__ nbr,
                                                          const float4 *__restrict__ g, const float4 *__restrict__ x4,
                                                          float w_rot, float w_reg, double *__restrict__ part)
{
    __shared__ double sh[NA_THREADS / 32];
    const int j = blockIdx.x * NA_THREADS + threadIdx.x;
    double er = 0.0, eg = 0.0;
    if (j < m) {
        const float *X = &x4[3 * j].x;
        const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {1, 2, 2, 0, 1, 2};
        for (int q = 0; q < 6; ++q) {
            float rho = X[pa[q]] * X[pb[q]] + X[4 + pa[q]] * X[4 + pb[q]] + X[8 + pa[q]] * X[8 + pb[q]];
            if (pa[q] == pb[q]) rho -= 1.0f;
            er += (double)w_rot * rho * rho;
        }
        const float4 gj = g[j];
        for (int s = 0; s < kg; ++s) {
            const int k = nbr[j * kg + s];
            if (k < 0) continue;
            const float4 gk = g[k];
            const float h[3] = {gk.x - gj.x, gk.y - gj.y, gk.z - gj.z};
            const float *xk = &x4[3 * k].x;
            for (int r = 0; r < 3; ++r) {
                const float e = ed_reg_residual(X + 4 * r, r, h, xk[4 * r + 3]);
                eg += (double)w_reg * e * e;
            }
        }
    }
    const double sr = na_block_sum(er, sh);
    const double sg = na_block_sum(eg, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sr;
        part[2 * blockIdx.x + 1] = sg;
    }
}

// the partial sums (lane k adds the CTAs k, k + 32, ... in order, then a
// fixed butterfly over the warp: deterministic), pose priors, six outputs
__global__ void __launch_bounds__(32) k_na_final(const double *__restrict__ pp, int np, const double *__restrict__ pn,
                                                 int nn, const double *__restrict__ pose, ed_solver_params prm,
                                                 double *__restrict__ out)
{
    const int lane = threadIdx.x;
    double ed = 0.0, erot = 0.0, ereg = 0.0, er = 0.0, ep = 0.0;
    for (int b = lane; b < np; b += 32) ed += pp[2 * b];
    for (int b = lane; b < nn; b += 32) {
        erot += pn[2 * b];
        ereg += pn[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ed += __shfl_xor_sync(0xffffffffu, ed, o);
        erot += __shfl_xor_sync(0xffffffffu, erot, o);
        ereg += __shfl_xor_sync(0xffffffffu, ereg, o);
    }
    if (lane != 0) return;
    for (int q = 0; q < 6; ++q) {
        const double d = pose[q] - prm.prior[q];
        if (q < 3) er += prm.w_r * d * d;
        else ep += prm.w_p * d * d;
    }
    out[0] = ed + erot + ereg + er + ep;
    out[1] = ed;
    out[2] = erot;
    out[3] = ereg;
    out[4] = er;
    out[5] = ep;
}

// device address of the scratch array: looked up afresh by every call made
// outside a stream capture (so a reloaded module after a device reset is
// found again); a call made during a capture, where the lookup may not run,
// takes the address the last call outside capture found
static std::mutex g_na_mutex;
static double *g_na_ptr[256];
static bool g_na_ready[256];

static ed_status na_scratch(cudaStream_t st, double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return ED_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();   // (e.g. the legacy stream queried while another stream captures)
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (cs == cudaStreamCaptureStatusNone || !g_na_ready[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "libed: ed_energy_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return ED_ERR_CUDA;
        }
        g_na_ptr[dev] = (double *)p;
        g_na_ready[dev] = true;
    }
    *out = g_na_ptr[dev];
    return ED_OK;
}

extern "C" ed_status ed_energy_noalloc(const float *pos, const float *nrm, const uint16_t *idx, const float *weights,
                                       int n_points, const float *nodes, const int *nbr, int m, int k_graph,
                                       const ed_frame *fr, const ed_solver_params *prm, const float *x,
                                       const double *pose, double *energy_out, cudaStream_t st)
{
    if (!pos || !nrm || !idx || !weights || !nodes || !nbr || !fr || !prm || !x || !pose || !energy_out ||
        n_points < 0 || m < 1 || k_graph < 1 || k_graph > ED_MAX_KG || !fr->depth || !fr->nmap ||
        fr->intr.width <= 0 || fr->intr.height <= 0)
        return ED_ERR_ARG;
    if (((uintptr_t)pos & 15) || ((uintptr_t)nrm & 15) || ((uintptr_t)weights & 15) || ((uintptr_t)nodes & 15) ||
        ((uintptr_t)x & 15) || ((uintptr_t)fr->nmap & 15) || ((uintptr_t)idx & 7))
        return ED_ERR_ARG;
    if (n_points > NA_MAX_POINTS || m > NA_MAX_NODES) {
        fprintf(stderr,
                "libed: ed_energy_noalloc: %d points / %d nodes exceed the fixed scratch of this entry point "
                "(at most %d points and %d nodes)\n",
                n_points, m, NA_MAX_POINTS, NA_MAX_NODES);
        return ED_ERR_CAPACITY;
    }
    double *scratch = nullptr;
    ed_status s = na_scratch(st, &scratch);
    if (s != ED_OK) return s;
    const int np = ed_div_up(n_points, NA_THREADS), nn = ed_div_up(m, NA_THREADS);
    double *pp = scratch, *pn = scratch + 2 * NA_MAX_POINT_CTAS;
    if (np > 0) {
        NaPointArgs a;
        a.pos = (const float4 *)pos;
        a.nrm = (const float4 *)nrm;
        a.w = (const float4 *)weights;
        a.g = (const float4 *)nodes;
        a.x4 = (const float4 *)x;
        a.idx = (const ushort4 *)idx;
        a.pose = pose;
        a.depth = fr->depth;
        a.nmap = (const float4 *)fr->nmap;
        a.K = fr->intr;
        a.n = n_points;
        a.eps2 = prm->eps_d * prm->eps_d;
        a.cos_eps_n = prm->cos_eps_n;
        a.sw = sqrtf(prm->w_data);
        a.part = pp;
        k_na_points<<<np, NA_THREADS, 0, st>>>(a); ed_note_launch();
    }
    k_na_nodes<<<nn, NA_THREADS, 0, st>>>(m, k_graph, nbr, (const float4 *)nodes, (const float4 *)x, prm->w_rot,
                                          prm->w_reg, pn); ed_note_launch();
    k_na_final<<<1, 32, 0, st>>>(pp, np, pn, nn, pose, *prm, energy_out); ed_note_launch();
    ED_LAUNCH_CHECK();
    return ED_OK;
}
