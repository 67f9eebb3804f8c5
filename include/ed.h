/*
 * ed.h -- C ABI of the B300 (sm_103a) embedded-deformation (ED) registration
 * hot path of MIS-SLAM (Song et al., "MIS-SLAM: Real-time Large Scale Dense
 * Deformable SLAM System in Minimal Invasive Surgery Based on Heterogeneous
 * Computing", arXiv 1803.02009).
 *
 * One frame of the path:
 *   ed_compute_normals  target normal map n(u)              (Sec. II.E, data term)
 *   ed_build_graph      ED nodes, k nearest nodes, weights,
 *                       node graph N(j)                     (Sec. II.D Eq. 1-2, Sec. II.E E_reg)
 *   ed_gn_step  x n_gn  warp + association + residuals + J^T J / J^T r
 *                       assembly + block-Jacobi PCG + update (Sec. II.E Eq. 3, Sec. II.F)
 *   ed_warp             final warp of every model point     (Sec. II.D Eq. 1; Sec. II.G)
 *   ed_fuse             registration map, Alg. 1 gate, fusion
 *                       Eqs. fusion1-4, lifting, deletion   (Sec. II.G, Alg. 1-3)
 *   ed_downsample       box averaging of the fused model    (Sec. III.A, Alg. 3)
 * and, for measurement, ed_depth_error (projected model minus depth, Sec. III).
 *
 * Conventions
 *   Units are millimetres.  Camera frame: x right, y down, z forward.
 *   Points and normals: float4 arrays [N][4]; points carry the fusion weight
 *   omega in w, normals carry the stability flag S in w.
 *   Node parameters x_j: the 3x4 affine [A_j | t_j] row-major, 12 floats per
 *   node: x[12j + 4r + c] = A_j[r][c] (c < 3), x[12j + 4r + 3] = t_j[r].
 *   Global pose: double[6] = (alpha, beta, gamma, Tx, Ty, Tz) with
 *   R = Rz(gamma) Ry(beta) Rx(alpha), warp v~ = R s + T (Eq. 1).
 *   Depth maps: float [H][W], 0 = hole.  Normal maps: float4 [H][W], w = 1
 *   valid / 0 invalid.  Colour maps: float4 [H][W].
 *
 * Ownership and errors
 *   The caller allocates every buffer; all pointers are device pointers unless
 *   a comment says host.  The library uses only the workspace handed to
 *   ed_create (size from ed_query_workspace) and never allocates device
 *   memory itself.  Every call is asynchronous on the given stream except
 *   where a comment says it synchronises.  A context must not be used from
 *   two streams at once.  Synchronous failures (bad arguments, launch
 *   errors) are returned as ed_status; conditions found on the device
 *   (non-finite values, PCG breakdown, capacity overflow, a timed-out wait)
 *   are written to the status word of ed_stats / ed_fuse's counts and to the
 *   context's device status word, readable after the stream synchronises.
 *   No kernel traps: every device wait is bounded.
 */
#ifndef ED_H_
#define ED_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ed_status {
    ED_OK = 0,
    ED_ERR_ARG = 1,        /* invalid argument (NULL, size, alignment, limits) */
    ED_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed */
    ED_ERR_CAPACITY = 3,   /* a size exceeded the limits the context was created with */
    ED_ERR_NONFINITE = 4,  /* a residual, energy or update was not finite */
    ED_ERR_BREAKDOWN = 5,  /* PCG found p^T H p <= 0 or a preconditioner block not SPD */
    ED_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    ED_ERR_STATE = 7       /* call order: e.g. ed_gn_step before ed_build_graph */
} ed_status;

/* Arithmetic of a Gauss-Newton step.  FP32: residuals, assembly and PCG in
 * FP32.  MIXED: FP32 residuals and assembly with two-sum compensated block
 * reductions, PCG dot products and norms accumulated as float-float
 * (about 44 significant bits, on the FP32 pipe), an FP64 master copy of the
 * node parameters that accumulates the updates.  MIXED_FP64: the same with
 * the PCG dot products and norms accumulated in FP64. */
enum { ED_PRECISION_FP32 = 0, ED_PRECISION_MIXED = 1, ED_PRECISION_MIXED_FP64 = 2 };
enum { ED_WEIGHT_GAUSSIAN = 0, ED_WEIGHT_EQ2 = 1 };

/* Capacities a context is created for; they size the workspace. */
typedef struct ed_limits {
    int max_points;          /* model points N */
    int max_nodes;           /* ED nodes m (<= 16384) */
    int max_width;           /* depth map size */
    int max_height;
    int max_pairs_per_node;  /* node pairs per node in J^T J (0 = 48) */
    int max_cells;           /* sampling grid cells (0 = 1 << 24) */
} ed_limits;

typedef struct ed_intrinsics {
    float fx, fy, cx, cy;    /* pinhole; pixel u covers [u - 0.5, u + 0.5) */
    int width, height;
} ed_intrinsics;

typedef struct ed_context ed_context;

/* Bytes of device workspace a context with these limits needs (host out). */
ed_status ed_query_workspace(const ed_limits *limits, size_t *bytes);

/* Creates a context on the current device over a caller-owned workspace of at
 * least ed_query_workspace bytes (256-byte aligned).  *ctx is a host handle. */
ed_status ed_create(const ed_limits *limits, void *workspace, size_t workspace_bytes, ed_context **ctx);
ed_status ed_destroy(ed_context *ctx);

/* Human-readable name of a status (static host string). */
const char *ed_status_string(ed_status s);

/*
 * Target normal map n(u) used by the point-to-plane data term (Sec. II.E:
 * "the corresponding normal to the pixel u").  The paper does not give the
 * operator; this library uses n = normalize((V(u,v+h) - V(u,v-h)) x
 * (V(u+h,v) - V(u-h,v))) over the back-projected depth V, oriented towards
 * the camera, invalid (all zero) when a stencil sample or the centre is a
 * hole or off the image.  depth [H][W] in, nmap [H][W][4] out.
 */
ed_status ed_compute_normals(ed_context *ctx, const float *depth, ed_intrinsics intr, int half_width,
                             float *nmap, cudaStream_t stream);

typedef struct ed_graph_params {
    int k;             /* nearest nodes per point; must be 4 (Eq. 1, "k nearest") */
    int k_graph;       /* node-graph neighbours |N(j)| (1..8) */
    int weight_mode;   /* ED_WEIGHT_GAUSSIAN: exp(-d^2/(2 sigma^2)); ED_WEIGHT_EQ2: 1 - d/d_max (Eq. 2) */
    float sigma;       /* Gaussian width (mm) */
    float node_radius; /* Poisson-disk radius (mm) when nodes are sampled */
    int max_nodes;     /* keep the first max_nodes sampled nodes (<= limits.max_nodes) */
    float search_cell; /* cell edge of the nearest-node search grid (mm); 0 = automatic */
} ed_graph_params;

/* Caller-owned device buffers of a deformation graph. */
typedef struct ed_graph {
    float *nodes;      /* [max_nodes][4] node positions g_j (input when m_in > 0) */
    uint16_t *idx;     /* [N][4] nearest nodes of each point, increasing distance */
    float *weights;    /* [N][4] normalised skinning weights */
    int *nbr;          /* [max_nodes][k_graph] node graph N(j) */
    int *counts;       /* int[4]: m (nodes in use), m_sampled (before truncation), nnzb, status */
} ed_graph;

/*
 * Builds the deformation graph of a model (Sec. II.D, II.E):
 *   nodes: the m_in given nodes when m_in > 0, else a phase-ordered
 *   Poisson-disk sample of the points with radius node_radius, truncated to
 *   max_nodes in selection order;
 *   skinning: the k nearest nodes of every point by the FP32 squared
 *   distance (ties to the lower node index), normalised weights (Eq. 1-2);
 *   node graph: the k_graph nearest other nodes of every node (alpha_jk = 1);
 *   and, internally, the block-sparsity pattern of J^T J, the points sorted
 *   by their set of four nodes and, per block, the runs of points that
 *   contribute to it, used by ed_gn_step.
 * pos/nrm [N][4] are the model (they must stay valid until the next
 * ed_build_graph); the graph buffers are retained by the context likewise.
 * The host waits twice, each time for an event queued early enough that the
 * GPU keeps working meanwhile (the grid sizes, queued before the Poisson
 * sampler's launch; the node count m, queued before the nearest-node search
 * and the tuple sort); everything after the node count -- the block pattern,
 * the incidences, the assembly's records -- is sized on the device, and the
 * call returns with it still queued.  The pattern's sizes (nnzb, runs) and the
 * PCG plan are read once, at the first later call that needs them
 * (ed_gn_step, ed_energy, ed_energy_grad, ed_graph_info asking for nnzb,
 * n_entries or n_runs, ed_batch_query_workspace); an error the build's
 * kernels report (ED_ERR_CAPACITY when the pattern exceeds max_nnzb,
 * ED_ERR_STATE for an inconsistent pattern) is returned by that call, and the
 * context has no graph afterwards.
 */
ed_status ed_build_graph(ed_context *ctx, const float *pos, const float *nrm, int n_points, int m_in,
                         const ed_graph_params *params, const ed_graph *graph, cudaStream_t stream);

/*
 * Sparse key correspondences (Sec. II.E "Correspondence"): the term
 * w_corr sum_k |v~_k - V_k|^2 over n_keypoints model key points kp_pos
 * (device [n][4], model frame, within the model's bounding box) warped by
 * Eq. (1) with the global pose, and their 3D targets kp_target (device
 * [n][4], camera frame of the new frame; w = 0 disables a key point).  The
 * paper's weight is w_corr = 10.  Call before ed_build_graph: the build then
 * skins the key points like model points (three rows per key point, after
 * the model points, so the graph's idx and weights must hold n_points +
 * 3 n_keypoints rows and max_points must cover them), and every later
 * ed_gn_step / ed_energy / ed_energy_grad includes the term (its energy in
 * ed_stats.e_corr and energy_out[6]).  The pointers are retained until the
 * next call; n_keypoints = 0 removes the term.
 */
ed_status ed_set_keypoints(ed_context *ctx, const float *kp_pos, const float *kp_target, int n_keypoints,
                           float w_corr);

/* Host-side sizes of the graph built last (host out; NULL entries skipped):
 * nodes m, stored 12x12 blocks nnzb (both triangles), the (block, point)
 * pairs the assembly visits per step (10 per point) and the runs of points
 * that share their four nearest nodes.  m alone is known when ed_build_graph
 * returns; asking for any of the others waits for the build's queued work
 * (and returns the build's error, if its kernels reported one). */
ed_status ed_graph_info(ed_context *ctx, int *m, int *nnzb, int *n_entries, int *n_runs);

typedef struct ed_frame {
    const float *depth;    /* [H][W] target depth D (mm), 0 = hole */
    const float *nmap;     /* [H][W][4] target normals from ed_compute_normals */
    const float *color;    /* [H][W][4] colour (ed_fuse only; may be NULL elsewhere) */
    ed_intrinsics intr;
} ed_frame;

typedef struct ed_solver_params {
    float w_data, w_rot, w_reg, w_r, w_p;  /* Eq. (3) weights (Sec. III.B: 1, 1000, 10000, 1e6, 1000) */
    float eps_d;           /* visible-point gate ||v~ - Gamma|| < eps_d (mm) */
    float cos_eps_n;       /* visible-point gate n~ . n(u) > cos_eps_n */
    int n_pcg;             /* PCG iterations per Gauss-Newton step */
    float pcg_tol;         /* early PCG stop when ||r|| <= tol ||b|| (0 = fixed count) */
    float lambda;          /* Levenberg-Marquardt damping: H + lambda diag(H) */
    float jitter;          /* preconditioner block shift, relative to trace/size */
    int precision;         /* ED_PRECISION_FP32, ED_PRECISION_MIXED or ED_PRECISION_MIXED_FP64 */
    double prior[6];       /* pose prior for E_r, E_p (Sec. II.E "Global Pose") */
    int lm_accept;         /* 1: Levenberg-Marquardt acceptance on the device (ed_lm_reset);
                              lambda then comes from the context's damping state */
} ed_solver_params;

/* Device-side statistics of one Gauss-Newton step, at its input (x, pose). */
typedef struct ed_stats {
    double energy;         /* Eq. (3) total */
    double e_data, e_rot, e_reg, e_rot_prior, e_pos_prior;
    double pcg_res0;       /* ||b|| */
    double pcg_res;        /* ||b - H d|| after the last PCG iteration */
    int n_valid;           /* points that passed the visible-point gate */
    int pcg_iters;
    int status;            /* ed_status of the device-side checks */
    int lm_rejected;       /* lm_accept: 1 when this step undid the previous one */
    double e_corr;         /* sparse key-correspondence energy (0 without key points) */
    double lambda;         /* damping of the system this step solved */
} ed_stats;

/*
 * One Gauss-Newton step of Eq. (3) (Sec. II.E-F): warp (Eq. 1), projective
 * association with the visible-point gate, data / rotation / regularisation
 * / pose-prior residuals, J^T J and J^T r assembled into 12x12 node blocks,
 * 6x12 pose-node blocks and a 6x6 pose block, then n_pcg iterations of
 * block-Jacobi preconditioned CG on (H + lambda diag H) d = -J^T r from d = 0,
 * and x += d, pose += d_pose.
 * x: [m][12] float, updated in place.  x_master: [m][12] double, required for
 * the mixed precisions (the master copy that accumulates the updates; x is
 * rewritten from it), ignored otherwise.  pose: double[6], updated in place.
 * stats: device ed_stats (may be NULL).  When a device check fails the
 * update is skipped and stats->status says why.  With params->lm_accept the
 * Levenberg-Marquardt decision of ed_lm_reset comes between the assembly and
 * the solve, and params->lambda is not used.
 */
ed_status ed_gn_step(ed_context *ctx, const ed_frame *frame, const ed_solver_params *params, float *x,
                     double *x_master, double *pose, ed_stats *stats, cudaStream_t stream);

/*
 * Start of a solve: x [m][12] = the identity warp (A_j = I, t_j = 0) for the
 * m nodes of the graph built last, x_master (may be NULL) the same in FP64,
 * pose double[6] = prior_host (host double[6]; NULL = zeros), in one launch
 * on the stream.
 */
ed_status ed_reset_params(ed_context *ctx, float *x, double *x_master, double *pose, const double *prior_host,
                          cudaStream_t stream);

/*
 * Levenberg-Marquardt damping schedule (Sec. II.F solves Eq. 3 with LM), kept
 * on the device so that a sequence of ed_gn_step calls needs no host
 * synchronisation and can be captured in a CUDA graph.  Steps with
 * params->lm_accept = 1 compare the energy at their input point with the
 * energy of the last accepted point: if it rose, the previous update is
 * undone (x, x_master, pose restored and the normal equations of the
 * accepted point reused, unchanged) and lambda <- 10 lambda (1e-4 when it
 * was 0); otherwise the point is accepted and lambda <- lambda / 10 (not on
 * the first step after a reset).  The system solved is H + lambda diag(H),
 * the block-Jacobi inverses taken from the damped diagonal blocks.  The
 * energy reported for a rejected step is that of the restored point.
 * ed_lm_reset starts a new solve: lambda = lambda0, no accepted point yet.
 * Enqueued on the stream; a context starts with lambda = 0 and no point, and
 * ed_build_graph forgets the accepted point (lambda is kept).
 */
ed_status ed_lm_reset(ed_context *ctx, float lambda0, cudaStream_t stream);

/*
 * Optional debug outputs of the next ed_gn_step calls (device buffers or
 * NULL): the warped points / normals and the associated pixel (v*W + u or
 * -1) of every model point, as computed inside the step.
 */
ed_status ed_set_debug(ed_context *ctx, float *warped_pos, float *warped_nrm, int *pix);

/*
 * Copies the assembled normal equations of the last ed_gn_step (device to
 * device): blocks [nnzb][12][12] in the row-major BSR order of row_ptr/col,
 * pose-node blocks [m][6][12], pose block [6][6], gradient J^T r [12m+6],
 * solution d [12m+6].  Any pointer may be NULL.  row_ptr [m+1], col [nnzb].
 */
ed_status ed_export_system(ed_context *ctx, int *row_ptr, int *col, float *blocks, float *pose_node,
                           float *pose_block, float *grad, float *delta, cudaStream_t stream);

/*
 * Limit of every bounded device-side wait in this context's launches (the
 * grid barriers of the PCG solve and of the node sampler, the look-back of
 * the library's scans, the waits for bulk copies into shared memory), in
 * nanoseconds of the GPU's global timer; 0 restores the default of 2 s.
 * Limits under 100 us are rejected (ED_ERR_ARG).  A wait that runs out sets
 * ED_ERR_TIMEOUT in the device status word (ed_stats.status of the step) and
 * the kernel returns; the PCG then leaves x and the pose unchanged.  Takes
 * effect for launches enqueued after the call.  The paper has no counterpart:
 * this is the bound that keeps a stalled launch from holding the GPU.
 */
ed_status ed_set_wait_limit(ed_context *ctx, unsigned long long limit_ns);

/*
 * Test hook for the bounded wait of the PCG grid barrier: the barrier of the
 * following ed_gn_step calls expects extra_arrivals (0..1024) more arrivals
 * than the launch has CTAs, so it can never complete and gives up after the
 * wait limit, reporting ED_ERR_TIMEOUT; 0 (the default) restores normal
 * operation.  The context stays usable.  The paper has no counterpart.
 */
ed_status ed_set_barrier_test(ed_context *ctx, int extra_arrivals);

/*
 * Measurement hook: from now on, record events[2k] / events[2k+1] (caller-
 * created cudaEvent_t, host array) on the launching stream immediately before
 * and after the k-th launch of the selected kernel, for k < n_pairs; the count
 * recorded so far goes to *recorded (host int, may be NULL).  kernel_id:
 * ED_KERNEL_PCG (the persistent PCG solve of ed_gn_step; in ed_batch_gn_step,
 * the batched PCG launch of each group, recorded on the group's first context),
 * ED_KERNEL_POINTS
 * (warp + association + residual pass and the compaction of its valid rows),
 * ED_KERNEL_ASSEMBLE (the block assembly and the diagonal blocks'
 * finalisation), ED_KERNEL_FINALIZE (the energy totals), ED_KERNEL_GRAD (the
 * per-node gradient kernel of ed_energy_grad).
 * n_pairs = 0 switches the hook off.  The paper has no counterpart: this is
 * instrumentation for roofline measurements.
 */
enum { ED_KERNEL_PCG = 0, ED_KERNEL_POINTS = 1, ED_KERNEL_ASSEMBLE = 2, ED_KERNEL_FINALIZE = 3, ED_KERNEL_GRAD = 4 };
ed_status ed_set_timing(ed_context *ctx, int kernel_id, cudaEvent_t *events, int n_pairs, int *recorded);

/*
 * The same hook sampled: of the selected kernel's launches i = 0, 1, ... from
 * now on, only those with i % every == every - 1 are recorded (pair k around
 * launch k * every + every - 1).  An event recorded between two kernels ends
 * their programmatic overlap, so a sampled hook keeps the other launches of a
 * timed loop undisturbed (every = the Gauss-Newton iterations of a frame
 * records the last PCG solve of every frame).  every >= 1 (ED_ERR_ARG
 * otherwise); ed_set_timing is every = 1.  Instrumentation; the paper has no
 * counterpart.
 */
ed_status ed_set_timing_every(ed_context *ctx, int kernel_id, cudaEvent_t *events, int n_pairs, int every,
                              int *recorded);

/* Kernel launches the library has issued in this process so far (host out).
 * Instrumentation; the paper has no counterpart. */
ed_status ed_launch_count(unsigned long long *count);

/*
 * Eq. (1) warp of n points with the graph built last:
 *   v~ = R sum_j w_j [A_j (v - g_j) + g_j + t_j] + T,
 *   n~ = normalize(R sum_j w_j A_j n).
 * pos_out.w = pos_in.w, nrm_out.w = nrm_in.w.
 */
ed_status ed_warp(ed_context *ctx, const float *x, const double *pose, const float *pos_in, const float *nrm_in,
                  int n_points, float *pos_out, float *nrm_out, cudaStream_t stream);

typedef struct ed_fuse_params {
    float tau_d;           /* Alg. 1: |z~ - D(u)| < tau_d (mm) */
    float cos_delta;       /* Alg. 1: n~ . n(u) > cos_delta */
    float omega_max;       /* Eq. fusion4 upper bound */
    int tau_time;          /* delete when frame - t > tau_time ... */
    float tau_weight;      /* ... and omega < tau_weight (Alg. 2 step 4, Alg. 3) */
    int frame;             /* current frame index (time stamp of fused / lifted points) */
} ed_fuse_params;

/*
 * Model update of Sec. II.G (Algorithms 1-3, Eqs. fusion1-4), out of place.
 * Inputs: the model (pos, nrm, col [n_in][4], t [n_in]) and the same points
 * warped into the frame (wpos, wnrm from ed_warp).  Reg keeps, per pixel, the
 * projected point with the smallest z~ (then the smallest index); a pixel is
 * registered when D(u) > 0, the normal is valid, |z~ - D(u)| < tau_d and
 * n~ . n(u) > cos_delta.  Registered points are fused with observation weight
 * 1 (moved along their ray to the fused depth, colour and normal averaged,
 * omega = min(omega + 1, omega_max), t = frame); every other valid pixel is
 * lifted as a new point (omega = 1, t = frame); unregistered old points with
 * frame - t > tau_time and omega < tau_weight are deleted.  Output order: kept
 * old points in their order, then lifted pixels in pixel order.
 * counts_out: device int[2] = (output count, status); the output is
 * truncated at capacity with status ED_ERR_CAPACITY.  reg_out ([H][W] point
 * index or -1) may be NULL.
 */
ed_status ed_fuse(ed_context *ctx, const float *pos, const float *nrm, const float *col, const int *tstamp,
                  int n_in, const float *wpos, const float *wnrm, const ed_frame *frame,
                  const ed_fuse_params *params, int capacity, float *pos_out, float *nrm_out, float *col_out,
                  int *t_out, int *counts_out, int *reg_out, cudaStream_t stream);

typedef struct ed_downsample_params {
    float box;             /* box edge (mm): the point-cloud density (Sec. III.A: 0.2 or 1 mm) */
    float omega_max;       /* cap of a merged point's fusion weight (Eq. fusion4) */
    float tau_weight;      /* stability flag of the merged point: omega >= tau_weight */
} ed_downsample_params;

/*
 * Box downsampling of a model (Sec. III.A: a fixed 3D box grid, the points in
 * each box averaged into one; Algorithm 3, first line), out of place.  The
 * boxes have edge params->box and are anchored at the minimum of the points'
 * bounding box; a point's box per axis is floor((x - min) / box) in FP32
 * (one subtraction, one IEEE division), boxes per axis floor((max - min) /
 * box) + 1, box key ix + nx (iy + ny iz).  The points of one box, taken in
 * increasing index order, become one point: omega-weighted means of position
 * and colour, the normalised omega-weighted sum of normals, weight
 * min(sum omega, omega_max), the latest time stamp, stability flag (nrm.w)
 * omega >= tau_weight; with no weight in a box, plain means.  Output in
 * increasing box key order.  Inputs as for ed_fuse; the outputs must not
 * alias the inputs.  counts_out: device int[2] = (output count, status); the
 * output is truncated at capacity with status ED_ERR_CAPACITY.  Returns
 * ED_ERR_CAPACITY when the grid has 2^32 boxes or more.  Synchronises the
 * stream once (it reads back the grid size to choose the sort's key width).
 */
ed_status ed_downsample(ed_context *ctx, const float *pos, const float *nrm, const float *col, const int *tstamp,
                        int n_in, const ed_downsample_params *params, int capacity, float *pos_out, float *nrm_out,
                        float *col_out, int *t_out, int *counts_out, cudaStream_t stream);

/*
 * Back-projection error (Sec. III measures the projected model image minus
 * the observed depth image).  The points wpos (device [n][4], in the frame's
 * camera frame, e.g. from ed_warp) are projected by the rule P of the
 * association; a pixel keeps the point of smallest z, then of lowest index.
 * Over the pixels that keep a point and have depth D > 0:
 * out (device double[4]) = (sum |z - D|, count, max |z - D|, sum (z - D)^2),
 * summed in a fixed order (deterministic).
 */
ed_status ed_depth_error(ed_context *ctx, const float *wpos, int n_points, const float *depth, ed_intrinsics intr,
                         double *out, cudaStream_t stream);

/*
 * Energy of Eq. (3) at (x, pose) with the graph built last (forward of the
 * differentiable warp + energy).  Association is recomputed and stored in
 * the context for ed_energy_grad.  energy_out has 7 entries when key points
 * are set (E_corr last) and 6 otherwise.  With Gaussian weights (the graph's
 * weight_mode) the skinning weights of Eq. (1) are recomputed from the node
 * indices instead of read from the graph (the same values, bit for bit), here
 * and in ed_energy_grad.  energy_out: device double[6] = (total,
 * data, rot, reg, rot prior, pos prior).
 */
ed_status ed_energy(ed_context *ctx, const ed_frame *frame, const ed_solver_params *params, const float *x,
                    const double *pose, double *energy_out, cudaStream_t stream);

/*
 * Gradient of Eq. (3) with respect to the node parameters and the pose,
 * with the association of the last ed_energy frozen: dE/dx [12m] and
 * dE/dpose [6] (float, device), scaled by grad_scale (the upstream gradient).
 * Written by its own kernels (per-point residual derivatives gathered per
 * node), independently of the J^T r assembly of ed_gn_step.
 */
ed_status ed_energy_grad(ed_context *ctx, const ed_frame *frame, const ed_solver_params *params,
                         const float *x, const double *pose, float grad_scale, float *grad_x, float *grad_pose,
                         cudaStream_t stream);

/*
 * The energy of ed_energy for callers that cannot allocate device memory
 * (host frameworks that own every device allocation and hand a plugin only
 * its buffers, real-time loops that forbid allocation after start-up).  The
 * paper has no counterpart: this is a deployment variant of ed_energy's
 * reduction.
 * It needs no context and no workspace: the caller passes the model (pos,
 * nrm [n][4]), its skinning (idx [n][4], weights [n][4]), the nodes [m][4],
 * the node graph nbr [m][k_graph], the frame, the parameters, x [m][12] and
 * the pose, and receives energy_out (device double[6]: total, data, rot, reg,
 * rot prior, pos prior).  The total is Eq. (3) without the key-correspondence
 * term E_corr (this entry point takes no key points): it equals ed_energy's
 * for a context with no key correspondences set.  The only scratch, the partial
 * sums of the reduction (133,120 bytes), is a fixed array in device global
 * memory inside the library, held by every GPU that loads it until the
 * process exits; no allocation routine is called.
 * Limits: n_points <= 2,097,152 and m <= 32,768; larger sizes return
 * ED_ERR_CAPACITY (with a message on stderr) before any launch.
 * Every call made outside a stream capture looks up the device address of
 * that array (cudaGetSymbolAddress, with the device current); a call made
 * during a capture takes the address that the last call outside capture
 * found, so make one plain call on the device before capturing (and again
 * after a device reset).  Every call writes every scratch slot it reads,
 * so stale contents never matter, but all calls share the one array: calls
 * that overlap on the GPU (different streams, or different host threads on
 * one device) race and must be serialised by the caller.
 */
ed_status ed_energy_noalloc(const float *pos, const float *nrm, const uint16_t *idx, const float *weights,
                            int n_points, const float *nodes, const int *nbr, int m, int k_graph,
                            const ed_frame *frame, const ed_solver_params *params, const float *x,
                            const double *pose, double *energy_out, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Batches of independent problems.
 *
 * Each problem is one frame of the registration of Sec. II (its own model,
 * node graph, depth map and pose prior) held in its own context, whose graph
 * has been built with ed_build_graph.  One batched Gauss-Newton iteration
 * does, for every problem, what ed_gn_step does (Eqs. 3-4 linearised, the
 * normal equations solved by block-Jacobi PCG, the update applied); it runs
 * the per-problem kernels up to the normal equations concurrently on
 * internal streams, the PCG solves of a group of problems as ONE persistent
 * cooperative launch in which each problem owns a range of CTAs with its own
 * grid barrier, then the updates.  The paper registers one frame at a time;
 * batching is a throughput variant of the same arithmetic.
 * ------------------------------------------------------------------------ */
typedef struct ed_batch ed_batch;

typedef struct ed_batch_schedule {
    int pcg_threads;          /* threads per PCG CTA: 512 (one CTA per SM) or 256 (two per SM) */
    int problems_per_launch;  /* problems sharing one persistent PCG launch (1..32); more
                                 problems per launch means fewer CTAs (more node rows) each */
    int streams;              /* internal streams for the per-problem kernels */
    int asm_blocks_per_warp;  /* off-diagonal 12x12 blocks per assembly warp: 2 (one per
                                 16-lane half) or 1 (the whole warp streams one block) */
    int point_chunk;          /* points per CTA of the step's point pass: 512 or 256 */
} ed_batch_schedule;

/*
 * Bytes of device workspace for a batch of `count` (1..64) problems: room
 * for a copy of every problem's x, x_master and pose (used by the autotuner).
 * Every context must hold a built graph (else ED_ERR_STATE).
 */
ed_status ed_batch_query_workspace(ed_context *const *ctxs, int count, size_t *bytes);

/*
 * Creates a batch over distinct contexts (ctxs[p] is problem p).  The caller
 * owns the contexts and the workspace (256-byte aligned, at least the queried
 * size), which must outlive the batch.  Creates `count` internal streams and
 * events (no device memory is allocated).  The default schedule is 512-thread
 * PCG CTAs, the largest power-of-two number of problems per launch whose CTA
 * shares fit in shared memory, min(count, 16) streams, two off-diagonal blocks
 * per assembly warp and 512 points per point-pass CTA.  A schedule's assembly
 * and point-pass choices are written into the member contexts (their own
 * ed_gn_step calls use them as well; a context starts with 2 and 512).  Rebuilding the
 * graph of a member context invalidates the batch: destroy and create it
 * again.  Returns ED_ERR_CAPACITY if no grouping fits.
 */
ed_status ed_batch_create(ed_context *const *ctxs, int count, void *workspace, size_t workspace_bytes,
                          ed_batch **batch);
ed_status ed_batch_destroy(ed_batch *batch);

/*
 * Sets the schedule (synchronises the device; drops a captured graph).
 * ED_ERR_ARG for a field outside its listed values; ED_ERR_CAPACITY if a
 * problem's CTA share does not fit in shared memory under it; the previous
 * schedule then stays in force.
 */
ed_status ed_batch_set_schedule(ed_batch *batch, const ed_batch_schedule *schedule);
ed_status ed_batch_get_schedule(const ed_batch *batch, ed_batch_schedule *schedule);

/*
 * One batched Gauss-Newton iteration, enqueued on `stream`.  Arrays of
 * `count` entries, indexed by problem: frames, params (all with the same
 * precision), x (device [m_p][12] float), x_master (host array of device
 * pointers, or NULL for FP32; entries required in mixed precision), pose
 * (device double[6]), stats (device ed_stats per problem, or NULL).  The host
 * arrays are read during the call only.  Same per-problem results and errors
 * as ed_gn_step; the block reductions of a batched PCG run over fewer CTAs,
 * so results agree with ed_gn_step to rounding, not bit for bit.
 */
ed_status ed_batch_gn_step(ed_batch *batch, const ed_frame *frames, const ed_solver_params *params,
                           float *const *x, double *const *x_master, double *const *pose, ed_stats *const *stats,
                           cudaStream_t stream);

/*
 * Captures n_iters batched iterations with these arguments into a CUDA graph
 * held by the batch (replacing any previous one); `stream` must be a created
 * stream, not the default one (ED_ERR_ARG); stats[p] then points to
 * n_iters consecutive ed_stats (one per iteration).  Nothing runs during the
 * capture.  The device buffers named here must stay valid while the graph
 * is replayed with ed_batch_launch, which enqueues all n_iters iterations
 * on `stream` with one graph launch.  ED_ERR_STATE from ed_batch_launch when
 * nothing was captured.
 */
ed_status ed_batch_capture(ed_batch *batch, const ed_frame *frames, const ed_solver_params *params,
                           float *const *x, double *const *x_master, double *const *pose, ed_stats *const *stats,
                           int n_iters, cudaStream_t stream);
ed_status ed_batch_launch(ed_batch *batch, cudaStream_t stream);

/*
 * Autotuner: times one captured batched iteration under every feasible PCG
 * schedule (PCG threads 512 / 256; problems per launch 1, 2, 4, ... up to
 * all; 4 or up to 16 streams) with the default assembly, then under the
 * assembly and point-pass choices (off-diagonal blocks per warp 2 / 1, points
 * per CTA 512 / 256) with the best PCG schedule, restoring every problem's x,
 * x_master and pose after each run, and keeps the fastest, returned in `chosen` (with its
 * time in ms in best_ms; either may be NULL).  Synchronises `stream` and the
 * device; drops a captured graph; `stream` must be a created stream.  Run it with the arguments of the real
 * iterations (the timings depend on the association of the current x).
 */
ed_status ed_batch_autotune(ed_batch *batch, const ed_frame *frames, const ed_solver_params *params,
                            float *const *x, double *const *x_master, double *const *pose, ed_stats *const *stats,
                            cudaStream_t stream, ed_batch_schedule *chosen, float *best_ms);

#ifdef __cplusplus
}
#endif

#endif /* ED_H_ */
