/*
 * cfd.h -- C ABI of the GB300 (sm_103a) implementation of the OpenCFD-SCU
 * stage right-hand side and TVD-RK3 step (arXiv:2209.15333).
 *
 * The library evaluates, on one GPU, the per-stage right-hand side
 *     L(U) = J * ( - sum_d delta_d fhat_d  +  sum_d D_d Fv_d )
 * of the curvilinear compressible Navier-Stokes equations (Eq. 1) with
 * Steger-Warming flux-vector splitting (Eqs. 19-30), UD7 / WENO7 / WENO5 or
 * hybrid reconstruction switched by the modified Jameson sensor
 * (Eq. 41-43, Section 2.2.3), masked-WENO5 boundary closures
 * (Section 2.2.4), 6th/8th-order central viscous terms (Eqs. 9-15,
 * Section 2.3) and the TVD Runge-Kutta update (Eq. 45).
 *
 * Conventions
 *  - Every call returns a cfd_status; nothing aborts, traps or throws.
 *  - Fields are double, structure-of-arrays [var][nz][ny][nx], xi (i)
 *    fastest.  Conserved variables U = (rho, rho u, rho v, rho w, E),
 *    nondimensional as in Eq. 17 (p = rho T/(gamma Ma^2)).
 *  - Pointers flagged on_device = 1 are device pointers on the context's
 *    device; they are read or written on the context's stream.  Host
 *    pointers are read or written before the call returns; pinned
 *    (page-locked, device-mapped) host buffers of the state are moved by
 *    the GPU's SMs through the mapped pointer, pageable ones by the copy
 *    engine.  Caller arrays stay caller-owned; the context copies what it
 *    keeps.
 *  - Directions without periodicity exclude nothing; periodic directions
 *    hold no duplicate end node.
 *  - A context is not thread-safe: use one context per host thread.
 *  - cfd_step is asynchronous.  Errors detected on the device (a
 *    non-physical state) surface as CFD_ENONPHYS from the next cfd_sync,
 *    cfd_get_state, cfd_rhs or cfd_step.
 */
#ifndef CFD_H
#define CFD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cfd_ctx cfd_ctx;

typedef enum {
    CFD_OK = 0,
    CFD_EINVAL = -1,        /* bad argument (message in cfd_last_error) */
    CFD_ENOMEM = -2,        /* device or host allocation failed */
    CFD_ECUDA = -3,         /* a CUDA runtime call failed */
    CFD_ENONPHYS = -4,      /* rho <= 0, p <= 0 or a NaN was met on the device */
    CFD_ETIMEOUT = -5,      /* cfd_sync gave up waiting */
    CFD_EUNSUPPORTED = -6   /* valid request the library does not implement */
} cfd_status;

/* boundary condition of one face (reading R12 of the paper's Table 8 case) */
enum {
    CFD_BC_PERIODIC = 0,        /* both faces of the direction must say so */
    CFD_BC_WALL_ISOTHERMAL = 1, /* u = 0 (+ blowing), T = T_wall, p_w = (4 p1 - p2)/3 */
    CFD_BC_INFLOW = 2,          /* Dirichlet from cfd_set_inflow (xi-low face) */
    CFD_BC_OUTFLOW_EXTRAP = 3,  /* zeroth-order extrapolation of primitives */
    CFD_BC_HALO = 4,            /* the first / last CFD_HALO_WIDTH layers are ghost layers that
                                   cfd_set_halo_links fills from a neighbouring block */
    CFD_BC_NONREFLECT = 5       /* characteristic non-reflecting boundary (the ramp case's
                                   "non-reflecting" outlet and top): linearised about the boundary
                                   node with the outward face normal grad(d)/|grad(d)|, the changes
                                   toward the first interior node of the entropy, shear and two
                                   acoustic variables are taken where the wave leaves the domain
                                   and dropped where it enters (Thompson 1987); supersonic outflow
                                   is zeroth-order extrapolation */
};

/* ghost layers per HALO face: the viscous terms reach 8 nodes (a central
   derivative of node fluxes that are central derivatives themselves) */
#define CFD_HALO_WIDTH 8

/* how the metrics argument of cfd_create is laid out */
enum {
    CFD_METRICS_3D = 0,       /* [10][nz][ny][nx] */
    CFD_METRICS_2D = 1,       /* [10][ny][nx], constant along zeta (extruded grids) */
    CFD_METRICS_UNIFORM = 2   /* [10], the same at every node */
};

enum { CFD_SUTHERLAND = 0, CFD_POWER = 1 };                 /* Eq. 15 / power law */
enum { CFD_UD7 = 0, CFD_WENO5 = 1, CFD_WENO7 = 2, CFD_HYBRID = 3 };  /* Table 2, Eq. 41-43 */
enum { CFD_METRIC_NODAL = 0, CFD_METRIC_FSP = 1 };
enum { CFD_FP64 = 0, CFD_FP32_BULK = 1 };
enum { CFD_SENSOR_PLAIN = 0, CFD_SENSOR_MLP = 1 };
enum { CFD_RECON_COMPONENT = 0, CFD_RECON_CHARACTERISTIC = 1 };  /* Sec. 2.2.2 */

typedef struct {
    int nx, ny, nz;            /* nodes per direction, each >= 1 (>= 8 if not periodic) */
    int bc_lo[3], bc_hi[3];    /* per direction xi, eta, zeta: CFD_BC_* */
    int metric_layout;         /* CFD_METRICS_* */
} cfd_grid;

typedef struct {
    double gamma, Re, Ma, Pr;  /* Re <= 0: inviscid (Eq. 17-18 parameters) */
    double T_wall;             /* nondimensional wall temperature */
    double T_ref;              /* reference temperature in K (Sutherland, Eq. 15) */
    int visc_law;              /* CFD_SUTHERLAND (S = 110.4 K) or CFD_POWER */
    double visc_omega;         /* power-law exponent: mu = T^omega */
    int scheme;                /* CFD_UD7, CFD_WENO5, CFD_WENO7, CFD_HYBRID */
    double theta1, theta2;     /* hybrid thresholds (paper: 0.02, 0.1) */
    int visc_order;            /* 6 or 8 */
    int metric_mode;           /* CFD_METRIC_NODAL (the paper: split fluxes with each node's own
                                  metrics), or CFD_METRIC_FSP: free-stream preserving -- every
                                  interface splits its eight stencil nodes with one interface
                                  metric, the 8-point midpoint interpolation of alpha = grad(d)/J
                                  (single-block contexts with periodic lines, component-wise
                                  reconstruction; a test and robustness mode) */
    int precision;             /* CFD_FP64 or CFD_FP32_BULK */
    int sensor;                /* CFD_SENSOR_PLAIN or CFD_SENSOR_MLP */
    double weno_eps;           /* epsilon of the WENO weights (1e-6) */
    int recon_vars;            /* CFD_RECON_COMPONENT, or CFD_RECON_CHARACTERISTIC: the WENO faces
                                  reconstruct characteristic fields (Eq. 31-40) -- the split fluxes
                                  of the stencil nodes projected with the left eigenvectors (Eq. 35)
                                  at the averaged state (Eq. 32) and the interface normal
                                  (alpha_j + alpha_{j+1})/|.|, mapped back with Eq. 34; UD7 faces
                                  are linear and stay component-wise */
} cfd_params;

/* cfd_params with the paper's defaults: gamma 1.4, Pr 0.72, theta 0.02/0.1,
   8th-order viscous terms, hybrid scheme, FP64, plain sensor, eps 1e-6,
   component-wise reconstruction. */
void cfd_default_params(cfd_params* p);

/*
 * Create a context on the current CUDA device.  metrics: xi_x, xi_y, xi_z,
 * eta_x, eta_y, eta_z, zeta_x, zeta_y, zeta_z, J (Eq. 3-4) in the layout
 * grid->metric_layout, host memory (metrics_on_device = 0) or device memory.
 * stream: a cudaStream_t, or NULL for a stream the context creates.
 * Allocates every device buffer the step needs (about 40 doubles per node
 * in FP64).  Errors: EINVAL (sizes -- every dimension >= 1, >= 8 on a
 * non-periodic line, ny and nz <= 65535, nx * ny < 2^31 -- BC pairs, params),
 * ENOMEM, ECUDA,
 * EUNSUPPORTED (FSP metric mode on non-periodic lines or with
 * characteristic reconstruction).
 */
cfd_status cfd_create(cfd_ctx** out, const cfd_grid* grid, const double* metrics,
                      int metrics_on_device, const cfd_params* params, void* stream);

/*
 * Ensemble of nblocks independent blocks of uneven sizes (grids[b],
 * metrics[b], params[b] for b < nblocks; every block may have its own gas
 * parameters, e.g. Ma and Re, but all share precision, scheme, viscous or
 * inviscid, visc_order and sensor).  cfd_step advances every block with one
 * persistent launch per kernel kind and stage (CTAs walk a work list of the
 * tiles of all blocks), captured with the boundary conditions as one CUDA
 * graph per RK3 step.  Per-block calls (cfd_set_state, cfd_get_state,
 * cfd_rhs, cfd_cfl_dt, cfd_get_flags) take the block index.  Not a step of
 * the paper itself: the single-GPU form of running many blocks at once.
 * Errors as cfd_create; CFD_EINVAL if the blocks disagree on shared settings.
 */
cfd_status cfd_create_batch(cfd_ctx** out, int nblocks, const cfd_grid* grids,
                            const double* const* metrics, int metrics_on_device,
                            const cfd_params* params, void* stream);

/*
 * Multi-block domains on one GPU (the single-GPU form of the paper's block
 * decomposition, Sec. 3): blocks of an ensemble exchange ghost layers.
 * links[(b * 3 + d) * 2 + side] is the block whose interior lies beyond face
 * (d, side) of block b, or -1.  A linked face must be CFD_BC_HALO; the grids
 * of the two blocks must agree in the two other directions (ghost layers
 * included), and a HALO direction needs at least 2 * CFD_HALO_WIDTH + 1
 * nodes.  Block b's ghost layers at the low face receive the neighbour's
 * layers [n - 2H, n - H), at the high face its layers [H, 2H) (H =
 * CFD_HALO_WIDTH), direction by direction (xi, then eta, then zeta, each
 * copying whole planes, so edges and corners are filled too).  The exchange
 * runs once here on the current states and, inside cfd_step, before every
 * RK3 stage; a block may be its own neighbour (periodic through ghosts).
 * Interior nodes then evolve exactly as in the undivided domain; ghost layers
 * of the state returned by cfd_get_state are stale.  links = NULL removes the
 * links.  Errors: CFD_EINVAL (not an ensemble, bad index, face not HALO,
 * size mismatch).
 */
cfd_status cfd_set_halo_links(cfd_ctx* ctx, const int* links);

/* Inflow profile for CFD_BC_INFLOW on the xi-low face: prim[5][ny] =
   rho, u, v, w, p per eta index, the same for every zeta (host memory). */
cfd_status cfd_set_inflow(cfd_ctx* ctx, const double* prim);

/* Wall-normal blowing/suction on the eta-low wall (reading R12):
   v_n = amp sin(2 pi (x-x0)/(x1-x0)) cos(2 pi m z/Lz) sin(omega t) for x in
   [x0, x1]; wall_x[nx], wall_z[nz] are the wall node coordinates (host). */
cfd_status cfd_set_blowing(cfd_ctx* ctx, double amp, double x0, double x1, double omega, int m,
                           double Lz, const double* wall_x, const double* wall_z);

/*
 * Learned shock sensor (not in the paper: it stands in for the sensor of
 * Eq. 42-43).  A 42 -> 32 -> 32 -> 3 MLP with ReLU, BF16 weights and FP32
 * accumulation on the tensor cores classifies every node (0 UD7, 1 WENO7,
 * 2 WENO5) from normalised stencil differences of p and rho (see
 * cfd_sensor_features); the interface rule (largest class over m-3..m+4)
 * applies as for the plain sensor.  A node whose largest softmax
 * probability is below conf_min, or whose features are not finite, takes
 * the plain sensor's class.  weights_bf16: W1[32][42], W2[32][32],
 * W3[3][32] (row = output), as consecutive bf16 (uint16) arrays; biases:
 * b1[32], b2[32], b3[3] float.  NULL weights switch back to the plain
 * sensor.  On an ensemble the weights apply to every block: one launch per
 * stage walks the zeta columns of all blocks, and cfd_sensor_fallbacks
 * counts the fallbacks of the ensemble's steps over all blocks.  The three
 * layers run per CTA on the tcgen05 tensor cores (accumulators in tensor
 * memory) or per warp with mma.sync: cfd_set_sweep_variant, dir 4.
 */
cfd_status cfd_set_sensor_mlp(cfd_ctx* ctx, const void* weights_bf16, const float* biases,
                              float conf_min);

/* The 42 sensor features of every node of the current state, float
   [42][nz][ny][nx]: for each direction d (xi, eta, zeta) and field q (p,
   rho), over line positions m-3..m+3 (periodic lines wrap, others clamp),
   (q_{m+t+1} - q_{m+t})/q_m for t = -3..2 and
   (q_{m-1} - 2 q_m + q_{m+1})/(q_{m-1} + 2 q_m + q_{m+1}); feature index
   (2 d + field) * 7 + t.  For training the learned sensor. */
cfd_status cfd_sensor_features(cfd_ctx* ctx, int block, float* out, int on_device);

/* Nodes that fell back to the plain sensor since the last call (reset). */
cfd_status cfd_sensor_fallbacks(cfd_ctx* ctx, unsigned long long* count);

/* Copy U [5][nz][ny][nx] into the context and apply the boundary
   conditions at the context time.  block: 0 (single-block contexts). */
cfd_status cfd_set_state(cfd_ctx* ctx, int block, const double* U, int on_device);

/* Copy the current state out. */
cfd_status cfd_get_state(cfd_ctx* ctx, int block, double* U, int on_device);

/* L(U) of the current state (one stage right-hand side, Eq. 44); zero on
   boundary nodes of non-periodic directions. */
cfd_status cfd_rhs(cfd_ctx* ctx, int block, double* dUdt, int on_device);

/* nsteps TVD-RK3 steps (Eq. 45) with a fixed dt; boundary conditions after
   every stage.  Replays a captured CUDA graph of one step. */
cfd_status cfd_step(cfd_ctx* ctx, double dt, int nsteps);

/* dt = cfl / max_n sum_d (|d_x u + d_y v + d_z w| + c |grad d|) of the
   current state (reading R16), computed on the device. */
cfd_status cfd_cfl_dt(cfd_ctx* ctx, int block, double cfl, double* dt);

/* Scheme class per node (0 UD7, 1 WENO7, 2 WENO5) of the last evaluation. */
cfd_status cfd_get_flags(cfd_ctx* ctx, int block, unsigned char* cls, int on_device);

/* Use these node classes instead of the sensor (cls = NULL: back to the
   sensor).  For comparing arithmetic with the hybrid switch held fixed. */
cfd_status cfd_force_flags(cfd_ctx* ctx, int block, const unsigned char* cls, int on_device);

/* Simulation time of the context (used by the blowing boundary condition). */
cfd_status cfd_get_time(cfd_ctx* ctx, double* t);
cfd_status cfd_set_time(cfd_ctx* ctx, double t);

/* Wait for the context's stream for at most timeout_s seconds: CFD_OK,
   CFD_ETIMEOUT (work still running; call again), CFD_ENONPHYS or CFD_ECUDA. */
cfd_status cfd_sync(cfd_ctx* ctx, double timeout_s);

/* Message of the last failure (never NULL; static storage if ctx is NULL). */
const char* cfd_last_error(const cfd_ctx* ctx);

/* Number of kernel launches issued by the context so far (all entry points). */
long long cfd_launch_count(const cfd_ctx* ctx);

/* Device probe, not a step of the method: measured dense FMA throughput of
   the current device in TFLOP/s (2 flops per FMA) for precision CFD_FP64 or
   CFD_FP32_BULK (float), used as the ALU roofline denominator.  Runs a
   fixed-length kernel of a few milliseconds on its own stream. */
cfd_status cfd_fma_peak(int precision, double* tflops);

/* Device self-check, not a step of the method.  The mixed-precision form
   converts between binary64 and binary32 with integer operations instead of
   the hardware cvt (which takes the narrow FP64 pipe); this runs those
   conversions against the hardware on the current device: float -> double on
   all 2^32 float bit patterns, double -> float (round to nearest even) on
   2^32 doubles from a fixed counter-based sequence that sweeps exponents
   across and around float's range and forces the rounding edges.  counts
   (host, CFD_CHECK_CONVERSIONS entries) receives: [0] floats checked,
   [1] float->double results differing from the hardware (NaN for NaN counts
   as equal), [2] doubles the integer path accepts, [3] their results
   differing from the hardware, [4] doubles whose acceptance disagrees with
   its range (zero, or 2^-126 <= |x| < 2^128).  A correct device gives
   [1] = [3] = [4] = 0.  Takes a few tens of milliseconds; CFD_EINVAL for a
   NULL counts, CFD_ECUDA on a CUDA error. */
#define CFD_CHECK_CONVERSIONS 5
cfd_status cfd_check_conversions(unsigned long long* counts);

/* Check entry, not a step of the method: the viscosity law of params
   (visc_law: Sutherland, Eq. 15, or the power law T^visc_omega) evaluated on
   the current device by the routine the viscous kernels use, in the
   arithmetic of params->precision (FP64, or FP32 for CFD_FP32_BULK: T is
   rounded to float first), at n temperatures.  T and mu are host arrays of
   n doubles.  The power law is table-driven (2^(e omega) m_k^omega times a
   binomial series in (m - m_k)/m_k, tables built from visc_omega on the
   host); temperatures outside [2^-64, 2^64), non-positive or not finite
   take exp(omega log T).  CFD_EINVAL for a bad argument or law, CFD_ECUDA
   on a CUDA error. */
cfd_status cfd_eval_viscosity(const cfd_params* params, const double* T, double* mu, int n);

/* Instrumentation, not a step of the method: run `reps` right-hand-side
   evaluations of the current state without a graph, with CUDA events between
   the kernels on the context stream, and return the mean milliseconds per
   evaluation of: [0] primitives, [1] sensor, [2] viscous fluxes,
   [3] xi sweep, [4] eta sweep, [5] zeta sweep (incl. J scaling).
   ms must hold CFD_PROFILE_KERNELS doubles. */
#define CFD_PROFILE_KERNELS 6
cfd_status cfd_profile_stage(cfd_ctx* ctx, int reps, double* ms);

/*
 * Allocation-free right-hand side.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code whose device
 * memory is owned by someone else (a framework's pool allocator or a fixed
 * memory budget, where an extra cudaMalloc fails or breaks the accounting)
 * and code that must not stall the device (cudaFree synchronises it).
 *
 * Computes the same L(U) as cfd_rhs for one block of at most
 * CFD_NOALLOC_MAX_NODES nodes, without a context: metrics (layout
 * grid->metric_layout), U [5][nz][ny][nx] and dUdt are DEVICE pointers
 * owned by the caller; the call is asynchronous on `stream` (a
 * cudaStream_t; NULL is the legacy default stream).  U is used as given: no
 * boundary conditions are applied to it.  All intermediate arrays live in
 * one fixed device array inside the library (about 14.5 MB, held by every
 * GPU that loads the library until the process exits); the call allocates
 * no device or host memory on success.
 *  - The first call on a device does a one-time set-up there (it looks up
 *    the array's device address and sets kernel attributes); make that
 *    first call before any stream capture.
 *  - Every call shares the one array and leaves its contents behind; calls
 *    that overlap on the GPU (several streams, several host threads) race.
 *    Order them on one stream.
 *  - Nothing detected on the device is reported (the call never
 *    synchronises with the host): neither a non-physical state nor, in the
 *    bounds-checked build, an out-of-range index; the next call clears the
 *    word that records them.  Check with cfd_rhs when that matters.
 * Errors: CFD_EINVAL (null pointer, bad grid or params), CFD_ENOMEM (the
 * grid has more than CFD_NOALLOC_MAX_NODES nodes), CFD_EUNSUPPORTED (FP32
 * bulk precision, characteristic reconstruction, the learned sensor -- it
 * has no weights here -- and what cfd_create rejects), CFD_ECUDA.
 */
#define CFD_NOALLOC_MAX_NODES 32768
cfd_status cfd_rhs_noalloc(const cfd_grid* grid, const cfd_params* params, const double* metrics,
                           const double* U, double* dUdt, void* stream);

/* Tuning control, not a step of the method.  The eta (dir 1) and zeta
   (dir 2) sweeps have three implementations with bit-identical results:
   kind 0 streams each x-row of 32 lanes along the line in segments of
   `param` nodes (one warp per row), kind 1 works on tiles of 32 x `param`
   (16 or 32) nodes with a 4-node halo that is split again in every tile,
   kind 2 walks segments of `param` nodes (0 = the whole line) with 8 warps
   in chunks of 8 positions, carrying the last stencil rows and face from
   chunk to chunk (no recomputation); kind 3 is kind 2 with the rows fetched
   by the tensor memory accelerator into a ring of staging buffers ahead of
   the warps (FP32 bulk only, nx a multiple of 32; CFD_EUNSUPPORTED
   otherwise).  dir 3 selects the xi sweep: kind 0 one CTA per 128-node
   segment with its halo, kind 1 walking segments of `param` nodes (0 = the
   whole line) in chunks of 128.  dir 0 selects the viscous node-flux
   kernel: kind 0 one thread per node reading its neighbours (CTAs along x
   rows), kind 1 / 2 a 32 x 8 tile streaming along zeta in segments of 64 /
   32 planes with a 9-plane shared ring, kind 3 as kind 0 with CTAs of 32 x 4
   nodes in x-y tiles (param ignored).  Ensembles offer three variants per
   kernel kind: viscous (2, 32), (1, 64), (3, 0); xi (0, 64), (0, 128),
   (1, 0); eta and zeta (1, 16), (1, 32), (2, 64).
   dir 4 selects the learned sensor's classifier (single contexts and
   ensembles; not tuned, and leaves the tuning alone): kind 0 runs the three
   layers per warp with mma.sync, kind 1 per CTA on the tcgen05 tensor cores
   with the accumulators in tensor memory (param ignored).  Single contexts
   use kind 1; an ensemble with the learned sensor times both on its first
   cfd_step and keeps the faster, unless one was fixed here.  The two forms add
   the biases at different points of the FP32 accumulation, so a logit can
   differ in its last bits between them.
   By default a context times the candidates on its first cfd_rhs / cfd_step
   and keeps the fastest; cfd_set_sweep_variant fixes one and turns the
   tuning off.  Choices are cached in the process and in a text file (the
   path in the environment variable CFD_GB300_TUNE_CACHE, "off" for none;
   default $XDG_CACHE_HOME or ~/.cache, paper_2209_15333_gb300/autotune.txt),
   keyed by library build, GPU name and SM count, precision, grid, boundary
   conditions and scheme, so that a later process skips the trial runs. */
cfd_status cfd_set_sweep_variant(cfd_ctx* ctx, int dir, int kind, int param);
cfd_status cfd_get_sweep_variant(cfd_ctx* ctx, int dir, int* kind, int* param);

/* Free every device buffer and the graph; NULL is allowed. */
void cfd_destroy(cfd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
