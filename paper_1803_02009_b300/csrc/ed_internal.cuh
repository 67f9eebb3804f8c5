// ed_internal.cuh -- context, workspace layout and device helpers of libed.
//
// Everything here is private to the library; the public ABI is include/ed.h.
#pragma once

#include <utility>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "ed.h"

#define ED_K 4                 // nearest nodes per point (Eq. 1)
#define ED_MAX_KG 8            // node-graph neighbours
#define ED_HARD_MAX_NODES 16384
#define ED_K1_THREADS 256
#define ED_K1_PART 32          // components of a point-kernel CTA partial (30 used)
#define ED_PCG_PART 16         // doubles per PCG CTA partial (at most)
#define ED_MAX_BATCH_LAUNCH 32 // problems in one batched PCG launch
#define ED_MAX_PCG_GRID 1184   // 8 x 148
#define ED_ASM_BINS 64         // incidence-count classes of the off-diagonal blocks (the last: 63 and more)
#define ED_PINNED_INTS (ED_MAX_PCG_GRID + 1 + 16)

// indices of the dmisc doubles: 0..7 energy terms of the current step
// (total, data, rot, reg, rot prior, pos prior, valid points, corr)
enum {
    DM_LAM = 16,         // Levenberg-Marquardt damping lambda
    DM_EPREV = 17,       // energy of the last accepted point
    DM_SAVED = 24,       // 24..31 energy terms of the last accepted point
    DM_POSE = 40,        // 40..45 from the pose pass: E_data, valid points, non-finite flag, E_corr, E_r, E_p
};

// indices of the misc int words in the workspace
enum {
    MI_STATUS = 0,       // device status word (ed_status)
    MI_M = 1,            // nodes in use
    MI_MTOTAL = 2,       // sampled nodes before truncation
    MI_DIMS = 4,         // 4..6 sampling-grid dims, 7 = cells
    MI_KDIMS = 8,        // 8..10 search-grid dims, 11 = cells
    MI_NNZB = 12,
    MI_SCAN_TOTAL = 13,
    MI_MAXSEG = 14,
    MI_NCHUNK = 15,
    MI_BBOX = 16,        // 16..21 ordered-int bbox (min xyz, max xyz)
    MI_PHASE_BASE = 24,  // running node count during sampling
    MI_BAR = 32,         // grid barrier arrival count of the PCG
    MI_BAR_GRAPH = 33,   // grid barrier arrival count of the Poisson sampler
    MI_LM_HAVE = 36,     // Levenberg-Marquardt: an accepted point is stored
    MI_LM_REJECT = 37,   // Levenberg-Marquardt: the current step undid the previous one
    MI_FUSE = 40,        // 40 kept, 41 lifted
    MI_READ = 48,        // 48..51 values gathered for one host read (chunk totals, upper blocks)
    MI_VOX = 52,         // 52..54 box-grid dims of ed_downsample, 55 its status
    MI_PHASES = 64,      // 64..90 phase counts, 96..123 starts, 128..154 fill counters
    MI_COUNT = 192
};
enum { MF_CELL = 0, MF_INV = 1, MF_KCELL = 2, MF_KINV = 3, MF_R2 = 4, MF_VOX = 5, MF_BBOX = 8, MF_COUNT = 16 };
// (MF_VOX .. MF_VOX + 2: the origin of the ed_downsample box grid)

// the mixed precisions (compensated reductions, FP64 master parameters)
static inline bool ed_is_mixed(int precision)
{
    return precision == ED_PRECISION_MIXED || precision == ED_PRECISION_MIXED_FP64;
}

// ordered-int image of a float (monotone for signed comparison)
__device__ __forceinline__ int f2o(float f)
{
    int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

// launch plan of the PCG of one problem
struct ed_pcg_plan_t {
    int grid;                // CTAs
    int nt;                  // threads per CTA (256 or 512)
    int ncache;              // blocks per CTA kept in shared memory
    int max_rows, max_blk;   // largest CTA share (rows, blocks)
    size_t smem;             // dynamic shared memory per CTA
};

// several problems in one persistent PCG launch
struct ed_pcg_batch_plan_t {
    int count, nt, grid;
    size_t smem;
    int cta_first[ED_MAX_BATCH_LAUNCH + 1];
    ed_pcg_plan_t plan[ED_MAX_BATCH_LAUNCH];
};

struct ed_context {
    ed_limits lim;
    char *ws;
    size_t ws_bytes;
    int device;
    int num_sms;

    // ---- workspace arrays ----
    int *misc;
    float *fmisc;
    double *dmisc;           // 64 doubles: pose-level scalars of the current step
    // sampling / search grids
    int *cell_of;            // [N]
    int *cell_pick;          // [cells]
    int *cell_node;          // [cells]
    int *kcell_start;        // [cells + 1]
    int *kcell_cnt;          // [cells]
    float4 *kcell_pos;       // [max_nodes] node positions by search cell (w: the node index as int bits)
    // pattern
    uint32_t *bitmap;        // [max_nodes * words]
    int bm_words;
    int *row_ptr;            // [max_nodes + 1]
    int *row_cnt;            // [max_nodes + 1]
    int *col;                // [max_nnzb]
    int *brow;               // [max_nnzb] row of each block
    int *tpos;               // [max_nnzb] position of the transposed block
    int *diag_pos;           // [max_nodes]
    int *up_list;            // [max_nnzb] upper block positions
    int4 *fin_info;          // [n_upper][2] packed assembly records (per frame, k_fin_pack)
    int max_nnzb;
    // the points in node-tuple order and the (block, run) incidences
    uint32_t *ent_key;       // [10 N] sort keys: tuple keys of the points, then the block of every incidence
    uint32_t *ent_val;       // [10 N] values: point indices of the tuple sort (and scratch of other sorts)
    uint32_t *ent_key2;      // radix temp
    uint32_t *ent_val2;
    int *radix_cnt;          // [256 * tiles + 1]
    uint32_t *inc;           // [10 N] incidences run << 4 | s << 2 | t sorted by block (kept for the frame)
    int *ent_start;          // [max_nnzb + 1] first incidence of every block
    int *perm;               // [N] point at each sorted position
    float4 *spos, *snrm;     // [N] positions and normals in sorted order
    ushort4 *sidx;           // [N] the tuple (nodes in increasing index order) at each sorted position
    float4 *sw;              // [N] skinning weights in tuple order
    ushort4 *sidx_d;         // [N] the nearest nodes in the graph's order (nearest first) at each sorted position
    float4 *sw_d;            // [N] their weights: the warp of a step sums in the order ed_warp and ed_energy do
    int *run_start;          // [N + 1] first sorted position of every run
    int *run_of_start;       // [N] r where sorted position k starts run r, else -1
    int *bcnt;               // [2 (max_nodes + 1)] bucket counts and fill counters of the tuple grouping
    int *bstart;             // [max_nodes + 1] bucket starts
    int *icnt;               // [2 (max_nnzb + 1)] incidence counts and fill counters per block
    int *asm_bins;           // [2 ED_ASM_BINS] off-diagonal blocks per incidence count, and fill counters (after icnt)
    // a step's valid rows, compacted in sorted order (k_compact)
    float4 *crec0, *crec1, *cpos, *csw;   // [N] records, position, tuple weights
    int *vrun_start;         // [N + 1] first compacted row of every run
    float *pose_R;           // [16] R of the step's pose (from the point pass)
    // normal equations
    float *bsr;              // [max_nnzb][144]
    float *grad;             // [12 m + 6] J^T r
    float *pnode;            // [m][72] pose-node blocks
    float *minv;             // [m][144] block-Jacobi inverses
    float *pose_blk;         // [36] pose block, [36..72) its inverse
    float *dmom;             // [m][72] moments (60) and J^T r (12) of the diagonal blocks, per step
    unsigned long long *lb_ticket;   // point pass of a step: epoch << 32 | chunks handed out
    unsigned long long *lb_state;    // [max_k1_ctas] per chunk: epoch << 34 | flag << 32 | valid rows
    // Levenberg-Marquardt: the undamped system and the parameters of the last
    // accepted point (restored when a step raises the energy)
    float *bsr_s;            // [max_nnzb][144]
    float *grad_s;           // [12 m + 6]
    float *pnode_s;          // [m][72]
    float *pblk_s;           // [36]
    float *x_prev;           // [m][12]
    double *xm_prev;         // [m][12]
    double *pose_prev;       // [6]
    float2 *node_energy;     // [m] (rot, reg) of every node
    int *pix;                // [N] association of the last evaluation
    float2 *k1_part;         // [ED_K1_PART][max_k1_ctas] float-float partials, component-major
    int max_k1_ctas;
    // PCG
    float *vec;              // 6 vectors of 12 max_nodes + 6: d, r, z, p0, p1, q
    size_t vec_stride;       // floats between vectors (multiple of 64: 16-byte aligned float4 rows)
    double *pcg_part;        // [2][ED_PCG_PART][ED_MAX_PCG_GRID] (component-major)
    double *red_part;        // [4][ED_MAX_PCG_GRID] per-CTA partials of ed_depth_error
    // fusion / scans
    unsigned long long *zbuf;  // [W H]
    int *regpix;             // [W H]
    int *fused_pix;          // [N]
    int *flag_a;             // [max(N, W H) + 1]
    int *flag_b;             // [max(N, W H) + 1]
    unsigned long long *scan_state;   // [scan_state_len] tile words of the one-pass scan
    int scan_state_len;
    unsigned *scan_ticket;   // tile ticket counter (never reset; host mirror below)
    unsigned scan_ticket_base, scan_epoch;
    float4 *gpts;            // [N] gradient per-point records (x2)
    float4 *comb_pos;        // [N] model points followed by the key-point rows (when key points are set)
    float4 *comb_nrm;

    // ---- graph state (host) ----
    int have_graph;
    int build_pending;       // the last build's pattern counts and PCG plan not read yet (ed_graph_ready)
    int asm_pairs;           // off-diagonal blocks per assembly warp (2, or 1 in a batch schedule)
    int pt_chunk;            // points per CTA of a step's point pass (512, or 256 in a batch schedule)
    // sparse key correspondences (ed_set_keypoints); rows n_model .. N of the
    // point set are the key points, three rows each
    const float4 *kp_pos, *kp_tgt;
    int n_kp;
    float w_corr;
    int n_model;
    const float *pos;
    const float *nrm;
    int N;
    ed_graph graph;
    int k_graph;
    int weight_mode;
    float sigma;
    int m;
    int nnzb;
    int n_upper;
    int n_entries;           // (block, point) pairs the assembly visits: 10 per point
    int n_runs;              // runs of equal node tuples
    int have_system;
    int have_energy;
    ed_pcg_plan_t pcg;       // single-problem PCG launch (one 512-thread CTA per SM)
    int *pcg_rows;           // [ED_MAX_PCG_GRID + 1] first node row of every CTA (device)
    int *pcg_rows_b;         // [ED_MAX_PCG_GRID + 1] the same for a batched launch (device)
    int *row_ptr_host;       // [max_nodes + 1] host copy of the block row pointer (pinned)
    int *pinned;             // [ED_PINNED_INTS] pinned host staging of small host-to-device copies

    // the pose pass of a Gauss-Newton step runs beside the assembly
    cudaStream_t aux;
    cudaEvent_t ev_fork, ev_join;
    // the misc words copied to the host without draining the stream
    int *misc_host;          // [MI_COUNT] pinned
    cudaEvent_t ev_misc;
    cudaEvent_t ev_build;    // the end of the last build's queued work (its copies to pinned memory)

    float *dbg_wpos, *dbg_wnrm;
    int *dbg_pix;

    // bounded device waits: limit (ed_set_wait_limit) and the extra arrivals
    // the PCG grid barrier expects (ed_set_barrier_test; 0 outside tests)
    unsigned long long wait_ns;
    int bar_extra;

    // measurement hook (ed_set_timing, ed_set_timing_every)
    int tm_kernel;
    cudaEvent_t *tm_events;
    int tm_pairs;
    int tm_count;
    int *tm_recorded;
    int tm_every;              // record launch i of the kernel when i % tm_every == tm_every - 1
    long long tm_seen;         // launches of the kernel since the hook was set
};

// events around one launch of a kernel selected by ed_set_timing
// a failed record switches the hook off and clears the error, so that it is
// never reported as the failure of a kernel launch
static inline void ed_tm_record(ed_context *c, cudaEvent_t e, cudaStream_t st)
{
    if (cudaEventRecord(e, st) != cudaSuccess) {
        (void)cudaGetLastError();
        fprintf(stderr, "libed: timing event record failed; timing hook disabled\n");
        c->tm_events = nullptr;
    }
}
// (an event between two kernels ends their programmatic overlap, so a
// sampled hook -- every tm_every-th launch -- leaves the others undisturbed)
static inline bool ed_tm_selected(const ed_context *c, int kid)
{
    return c->tm_events && c->tm_kernel == kid && c->tm_count < c->tm_pairs &&
           c->tm_seen % c->tm_every == c->tm_every - 1;
}
static inline void ed_tm_begin(ed_context *c, int kid, cudaStream_t st)
{
    if (ed_tm_selected(c, kid)) ed_tm_record(c, c->tm_events[2 * c->tm_count], st);
}
static inline void ed_tm_end(ed_context *c, int kid, cudaStream_t st)
{
    if (!c->tm_events || c->tm_kernel != kid) return;
    if (ed_tm_selected(c, kid)) {
        ed_tm_record(c, c->tm_events[2 * c->tm_count + 1], st);
        if (!c->tm_events) return;
        c->tm_count++;
        if (c->tm_recorded) *c->tm_recorded = c->tm_count;
    }
    c->tm_seen++;
}

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------

#define ED_CUDA_TRY(call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            fprintf(stderr, "libed: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                                 \
            return ED_ERR_CUDA;                                                                \
        }                                                                                      \
    } while (0)

#define ED_LAUNCH_CHECK()                                                                      \
    do {                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess) {                                                               \
            fprintf(stderr, "libed: launch failed: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return ED_ERR_CUDA;                                                                \
        }                                                                                      \
    } while (0)

static inline int ed_div_up(long a, long b) { return (int)((a + b - 1) / b); }

// process-wide count of kernel launches issued by the library (host side)
void ed_note_launch();
void ed_note_launches(unsigned long long n);   // kernels of a replayed CUDA graph

// ---------------------------------------------------------------------------
// exact FP32 decision rules (no fused multiply-add, fixed operation order)
// ---------------------------------------------------------------------------

// squared distance key dx*dx + dy*dy + dz*dz, left to right
__device__ __forceinline__ float ed_key(float px, float py, float pz, float gx, float gy, float gz)
{
    float dx = __fsub_rn(px, gx);
    float dy = __fsub_rn(py, gy);
    float dz = __fsub_rn(pz, gz);
    float s = __fmul_rn(dx, dx);
    s = __fadd_rn(s, __fmul_rn(dy, dy));
    s = __fadd_rn(s, __fmul_rn(dz, dz));
    return s;
}

__device__ __forceinline__ float ed_dot3_exact(float ax, float ay, float az, float bx, float by, float bz)
{
    float s = __fmul_rn(ax, bx);
    s = __fadd_rn(s, __fmul_rn(ay, by));
    s = __fadd_rn(s, __fmul_rn(az, bz));
    return s;
}

// P(v): q = x / z, t = fx q, t += cx, t += 0.5, pixel = floor(t)
__device__ __forceinline__ bool ed_project(float x, float y, float z, const ed_intrinsics &K, int &u, int &v)
{
    if (!(z > 0.0f)) return false;
    float tx = __fadd_rn(__fadd_rn(__fmul_rn(K.fx, __fdiv_rn(x, z)), K.cx), 0.5f);
    float ty = __fadd_rn(__fadd_rn(__fmul_rn(K.fy, __fdiv_rn(y, z)), K.cy), 0.5f);
    float fu = floorf(tx), fv = floorf(ty);
    if (!(fu >= 0.0f && fu < (float)K.width && fv >= 0.0f && fv < (float)K.height)) return false;
    u = (int)fu;
    v = (int)fv;
    return true;
}

// Pi(u, D) for the gates: ((u - cx) D / fx, (v - cy) D / fy, D)
__device__ __forceinline__ float3 ed_backproject(int u, int v, float D, const ed_intrinsics &K)
{
    float a = __fdiv_rn(__fmul_rn(__fsub_rn((float)u, K.cx), D), K.fx);
    float b = __fdiv_rn(__fmul_rn(__fsub_rn((float)v, K.cy), D), K.fy);
    return make_float3(a, b, D);
}

// ---------------------------------------------------------------------------
// global pose
// ---------------------------------------------------------------------------

struct ed_pose_f {
    float R[9];
    float dR[27];   // dR/dalpha, dR/dbeta, dR/dgamma
    float T[3];
};

__device__ __forceinline__ void ed_mat3_mul_f(const float *a, const float *b, float *c)
{
    float t[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) t[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
#pragma unroll
    for (int i = 0; i < 9; ++i) c[i] = t[i];
}

// R = Rz(gamma) Ry(beta) Rx(alpha) and its angle derivatives in FP32 (one
// thread per CTA; the results are FP32 matrices in any case)
__device__ inline void ed_pose_eval(const double *pose, ed_pose_f &P)
{
    float sa, ca, sb, cb, sg, cg;
    sincosf((float)pose[0], &sa, &ca);
    sincosf((float)pose[1], &sb, &cb);
    sincosf((float)pose[2], &sg, &cg);
    const float Rx[9] = {1, 0, 0, 0, ca, -sa, 0, sa, ca}, dRx[9] = {0, 0, 0, 0, -sa, -ca, 0, ca, -sa};
    const float Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb}, dRy[9] = {-sb, 0, cb, 0, 0, 0, -cb, 0, -sb};
    const float Rz[9] = {cg, -sg, 0, sg, cg, 0, 0, 0, 1}, dRz[9] = {-sg, -cg, 0, cg, -sg, 0, 0, 0, 0};
    float t[9];
    ed_mat3_mul_f(Rz, Ry, t);
    ed_mat3_mul_f(t, Rx, P.R);
    ed_mat3_mul_f(t, dRx, P.dR);
    ed_mat3_mul_f(Rz, dRy, t);
    ed_mat3_mul_f(t, Rx, P.dR + 9);
    ed_mat3_mul_f(dRz, Ry, t);
    ed_mat3_mul_f(t, Rx, P.dR + 18);
    for (int i = 0; i < 3; ++i) P.T[i] = (float)pose[3 + i];
}

// ---------------------------------------------------------------------------
// Eq. (1) warp of one point (shared by ed_warp, the GN step and the gradient)
// ---------------------------------------------------------------------------

struct ed_warped {
    float3 s;     // sum_j w_j [A_j (v - g_j) + g_j + t_j] (before the global pose)
    float3 v;     // R s + T
    float3 n;     // normalize(R sum_j w_j A_j n)
};

// ---------------------------------------------------------------------------
// programmatic dependent launch: a kernel launched by ed_launch_pdl may be
// dispatched while the kernel before it on the stream is still finishing; it
// calls ed_pdl_wait() before it reads or writes anything that kernel touches
// (launched without the attribute, the wait returns at once).  Only for a
// kernel whose stream predecessor is a kernel: not after a wait on another
// stream's event.  Reads before the wait are limited to data written two or
// more kernels back by kernels that call ed_pdl_trigger after their own wait.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ed_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// lets the next programmatic dependent launch start (its CTAs fill the slots
// this kernel frees); called after ed_pdl_wait, so that a dependent may read,
// before its own wait, anything written two or more kernels back
__device__ __forceinline__ void ed_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static inline cudaError_t ed_launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                        Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ed_launch_pdl with no dynamic shared memory, returning from the enclosing
// ed_status function on a launch error (the kernel starts with ed_pdl_wait)
#define ED_LAUNCH(kern, grid, block, st, ...) \
    ED_CUDA_TRY(ed_launch_pdl(kern, dim3(grid), dim3(block), 0, st, __VA_ARGS__))

// a cooperative launch (co-resident CTAs), as a programmatic dependent launch
// when pdl is set (the kernel then starts with ed_pdl_wait)
static inline cudaError_t ed_launch_coop(const void *fn, int grid, int nt, void **args, size_t smem, cudaStream_t st,
                                         bool pdl)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ---------------------------------------------------------------------------
// grid barrier of a cooperative (co-resident) launch, with a bounded wait
// ---------------------------------------------------------------------------

#define ED_BAR_TIMEOUT_NS 2000000000ull   // default limit of a device wait (ed_set_wait_limit)
#define ED_MIN_WAIT_NS 100000ull          // shortest limit ed_set_wait_limit accepts (100 us)

__device__ __forceinline__ unsigned long long ed_gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ed_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ed_atom_add_release(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void ed_st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ed_ld_acquire64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void ed_st_release64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void ed_red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// grid barrier on a monotonic arrival counter that every CTA polls: the CTA's
// writes happen before thread 0's arrival through the CTA barrier, and the
// arrival is a release (cumulative over that happens-before: no separate
// fence, which cost about 0.17 us per barrier); other CTAs' writes are visible
// after its acquire load of the count and the CTA barrier that follows (later
// reads of shared data bypass L1); returns false when the context status is
// set (an error elsewhere, or this wait timed out)
__device__ __forceinline__ bool ed_grid_sync(unsigned *count, int *status, unsigned nblocks, unsigned &target, int *s_flag,
                                             unsigned long long limit_ns = ED_BAR_TIMEOUT_NS)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += 1;
        ed_red_add_release(count, 1u);
        const unsigned goal = nblocks * target;
        const unsigned long long t0 = ed_gtimer();
        unsigned spins = 0;
        while (ed_ld_acquire(count) < goal) {
            if ((++spins & 63u) == 0) {
                if (*(volatile int *)status != ED_OK) { ok = 0; break; }
                if (ed_gtimer() - t0 > limit_ns) {
                    atomicCAS(status, ED_OK, ED_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}


// ---------------------------------------------------------------------------
// bulk asynchronous global -> shared copies completing on an mbarrier
// (addresses and sizes 16-byte aligned)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ed_smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ed_mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ed_smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the calling thread arrives and announces `bytes` of copies to come
__device__ __forceinline__ void ed_mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ed_smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void ed_bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     ed_smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(ed_smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool ed_mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(ed_smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait for phase `parity` of an mbarrier (all threads may call it);
// false when limit_ns passed (the caller records the error and then waits
// once more for its copies before leaving)
__device__ __forceinline__ bool ed_mbar_wait(unsigned long long *bar, unsigned parity,
                                             unsigned long long limit_ns = ED_BAR_TIMEOUT_NS)
{
    const unsigned long long t0 = ed_gtimer();
    while (!ed_mbar_test(bar, parity))
        if (ed_gtimer() - t0 > limit_ns) return false;
    return true;
}

// Float-float accumulation (value = hi + lo): Knuth's error-free two-sum of
// the high parts, the low parts added to its error, then a fast two-sum
// renormalisation.  About 44 significant bits on the FP32 pipe (B300's FP64
// rate is a small fraction of its FP32 rate); deterministic for a fixed order.
__device__ __forceinline__ float2 ed_ff_add(float2 a, float2 b)
{
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    const float lo = __fadd_rn(err, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(s, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

__device__ __forceinline__ float2 ed_ff_add1(float2 a, float b) { return ed_ff_add(a, make_float2(b, 0.f)); }

__device__ __forceinline__ double ed_ff_value(float2 a) { return (double)a.x + (double)a.y; }

// butterfly sum of one float-float value over the warp (lane 0's result is
// the one used: a fixed pattern, so it is deterministic)
__device__ __forceinline__ float2 ed_ff_warp_sum(float2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float2 u = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
        v = ed_ff_add(v, u);
    }
    return v;
}

// Eq. (1) skinning weights, Gaussian mode, from the keys of the k = 4
// nearest nodes (slots >= nvalid hold no node): w~_s = exp(-d_s^2 / 2 sigma^2),
// normalised to sum 1 (1/4 each if all vanish).  Graph build and the
// recomputation in the energy / gradient path both use this function, so
// recomputed weights equal the stored ones bit for bit.
__device__ __forceinline__ float4 ed_gauss_weights_from_keys(const float *kk, int nvalid, float sigma)
{
    float w[4], sum = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float t = s < nvalid ? expf(-kk[s] / (2.0f * sigma * sigma)) : 0.f;
        if (!(t > 0.f)) t = 0.f;
        w[s] = t;
        sum += t;
    }
    const float inv = sum > 0.f ? 1.0f / sum : 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) w[s] = sum > 0.f ? w[s] * inv : 0.25f;
    return make_float4(w[0], w[1], w[2], w[3]);
}

// the same weights recomputed from a point and its node indices
__device__ __forceinline__ float4 ed_gauss_weights(float4 p, ushort4 id, const float4 *__restrict__ g, int m,
                                                   float sigma)
{
    const unsigned short ids[4] = {id.x, id.y, id.z, id.w};
    float kk[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float4 gs = __ldg(g + ids[s]);
        kk[s] = ed_key(p.x, p.y, p.z, gs.x, gs.y, gs.z);
    }
    return ed_gauss_weights_from_keys(kk, m < 4 ? m : 4, sigma);
}

__device__ __forceinline__ ed_warped ed_warp_point(float4 p, float4 nr, ushort4 id, float4 w, const float4 *__restrict__ g,
                                                    const float4 *__restrict__ x4, const float *R, const float *T)
{
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
    const unsigned short ids[4] = {id.x, id.y, id.z, id.w};
    const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = ids[k];
        const float4 gj = __ldg(g + j);
        const float4 a0 = __ldg(x4 + 3 * j), a1 = __ldg(x4 + 3 * j + 1), a2 = __ldg(x4 + 3 * j + 2);
        const float dx = p.x - gj.x, dy = p.y - gj.y, dz = p.z - gj.z;
        const float wk = ws[k];
        s0 += wk * (a0.x * dx + a0.y * dy + a0.z * dz + a0.w + gj.x);
        s1 += wk * (a1.x * dx + a1.y * dy + a1.z * dz + a1.w + gj.y);
        s2 += wk * (a2.x * dx + a2.y * dy + a2.z * dz + a2.w + gj.z);
        n0 += wk * (a0.x * nr.x + a0.y * nr.y + a0.z * nr.z);
        n1 += wk * (a1.x * nr.x + a1.y * nr.y + a1.z * nr.z);
        n2 += wk * (a2.x * nr.x + a2.y * nr.y + a2.z * nr.z);
    }
    ed_warped o;
    o.s = make_float3(s0, s1, s2);
    o.v = make_float3(R[0] * s0 + R[1] * s1 + R[2] * s2 + T[0], R[3] * s0 + R[4] * s1 + R[5] * s2 + T[1],
                      R[6] * s0 + R[7] * s1 + R[8] * s2 + T[2]);
    float m0 = R[0] * n0 + R[1] * n1 + R[2] * n2;
    float m1 = R[3] * n0 + R[4] * n1 + R[5] * n2;
    float m2 = R[6] * n0 + R[7] * n1 + R[8] * n2;
    float l2 = m0 * m0 + m1 * m1 + m2 * m2;
    float il = l2 > 0.f ? 1.0f / sqrtf(l2) : 0.f;
    o.n = make_float3(m0 * il, m1 * il, m2 * il);
    return o;
}

// E_reg residual of an edge j -> k, row r: A_j (g_k - g_j) + g_j + t_j - g_k - t_k,
// evaluated as (A_j - I)(g_k - g_j) + t_j - t_k (identical algebra) so that no
// term of the size of the coordinates (~60 mm) cancels in FP32.
// xrow = row r of [A_j | t_j]; h = g_k - g_j; tk = t_k[r].
__device__ __forceinline__ float ed_reg_residual(const float *xrow, int r, const float *h, float tk)
{
    float a0 = xrow[0], a1 = xrow[1], a2 = xrow[2];
    if (r == 0) a0 -= 1.0f;
    else if (r == 1) a1 -= 1.0f;
    else a2 -= 1.0f;
    return a0 * h[0] + a1 * h[1] + a2 * h[2] + (xrow[3] - tk);
}

// association of a warped point: pixel index or -1 (visible-point gate, Sec. II.E)
__device__ __forceinline__ int ed_associate(const ed_warped &W, const float *__restrict__ depth,
                                            const float4 *__restrict__ nmap, const ed_intrinsics &K, float eps2,
                                            float cos_eps_n)
{
    int u, v;
    if (!ed_project(W.v.x, W.v.y, W.v.z, K, u, v)) return -1;
    const int q = v * K.width + u;
    const float D = __ldg(depth + q);
    if (!(D > 0.0f)) return -1;
    const float4 tn = __ldg(nmap + q);
    if (tn.w == 0.0f) return -1;
    const float3 G = ed_backproject(u, v, D, K);
    const float dx = __fsub_rn(W.v.x, G.x), dy = __fsub_rn(W.v.y, G.y), dz = __fsub_rn(W.v.z, G.z);
    if (!(ed_dot3_exact(dx, dy, dz, dx, dy, dz) < eps2)) return -1;
    if (!(ed_dot3_exact(W.n.x, W.n.y, W.n.z, tn.x, tn.y, tn.z) > cos_eps_n)) return -1;
    return q;
}

// ---------------------------------------------------------------------------
// internal entry points shared between translation units
// ---------------------------------------------------------------------------

// the counts and PCG plan of the last build (one host wait at the first call
// after the build that needs them); ED_ERR_STATE without a graph
ed_status ed_graph_ready(ed_context *ctx, cudaStream_t st);

// exclusive scan of n ints (out[n] = the total, also stored to *total2 when
// given); with n_dev, of *n_dev ints, the length read on the device (none
// when it exceeds n, the capacity the launch is sized for)
ed_status ed_scan_exclusive(ed_context *ctx, const int *in, int *out, int n, cudaStream_t st,
                            int *total2 = nullptr, const int *n_dev = nullptr);
ed_status ed_radix_sort_pairs(ed_context *ctx, uint32_t *keys, uint32_t *vals, int n, int key_bits, cudaStream_t st);
ed_status ed_bbox_enqueue(ed_context *ctx, const float4 *pos, int n, cudaStream_t st);
ed_status ed_pcg_solve(ed_context *ctx, const ed_solver_params *prm, float *x, double *xm, double *pose,
                       ed_stats *stats, cudaStream_t st);
ed_status ed_pcg_plan(ed_context *ctx, const int *row_ptr_host, cudaStream_t st);
ed_status ed_gn_pre(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, float *x, double *x_master,
                    double *pose, ed_stats *stats, cudaStream_t st, bool fork_pose = true);
ed_status ed_gn_post(ed_context *ctx);
ed_status ed_pcg_make_plan(const int *row_ptr_host, int m, int grid, int nt, ed_pcg_plan_t *pl, int *rows_start);
ed_status ed_pcg_batch_plan(ed_context *const *ctxs, int count, int nt, int grid_total, ed_pcg_batch_plan_t *bp);
ed_status ed_pcg_solve_batch(ed_context *const *ctxs, const ed_pcg_batch_plan_t *bp, const ed_solver_params *const *prm,
                             float *const *x, double *const *xm, double *const *pose, ed_stats *const *stats,
                             cudaStream_t st);
ed_status ed_point_pass(ed_context *ctx, const ed_frame *fr, const ed_solver_params *prm, const float *x,
                        const double *pose, int write_records, cudaStream_t st);
