// cfd_api.cu -- the C ABI (include/cfd.h): context, device buffers, stage
// orchestration and CUDA-graph replay of the TVD-RK3 step (Eq. 45).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>

#include <sys/stat.h>

#include "../../include/cfd.h"
#include "cfd_kernels.cuh"

using namespace cfdk;

namespace {

constexpr int kSMs = 152;
// kernel kinds of an ensemble with more than one variant, the number of
// variants each, and the walking eta/zeta segment of the ensemble
enum { KIND_VISC = 0, KIND_SX = 1, KIND_T1 = 2, KIND_T2 = 3, KIND_COUNT = 4 };
constexpr int kBatchVariants = 3;
constexpr int kBatchWS = 64;
// work-list maps of an ensemble, one per kernel kind and variant (see
// batch_tiles), and the learned sensor's zeta columns
enum {
    MAP_NODE = 0,
    MAP_VISC = 1,  // + variant (3)
    MAP_SX = 4,    // + variant (3)
    MAP_T1 = 7,    // + variant (3)
    MAP_T2 = 10,   // + variant (3)
    MAP_MLP = 13,
    MAP_COUNT = 14
};
constexpr int kBatchMlpTZ = 16;  // planes per zeta segment of the ensemble's learned sensor

struct Bufs {
    double* U = nullptr;      // [5][N] state U^n
    double* Uk = nullptr;     // [5][N] stage state
    void* P = nullptr;        // [7][N] primitives
    void* Fv = nullptr;       // [12][N] viscous fluxes
    void* R = nullptr;        // [5][N] accumulator
    uint8_t* cls = nullptr;   // [N]
    uint8_t* cls_tune = nullptr;  // [N] class buffer of the autotuner's trial runs
};

}  // namespace

struct cfd_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cfd_grid grid{};
    cfd_params prm{};
    Geo g{};
    Phys ph{};
    BCData bc{};
    Bufs b;
    double* met = nullptr;          // [31][M]
    float* metf = nullptr;          // [31][M] float mirror
    int sweep_kind[3] = {0, 0, 0};  // eta/zeta: 0 streaming, 1 tile, 2 walking (chosen by the autotuner)
    int sweep_param[3] = {0, 128, 128};
    int xi_kind = 1;                // xi: 0 one CTA per segment of bx nodes with its halo, 1 walking
    int xi_seg = 0;                 // walking xi: nodes per CTA (0 = the whole line)
    int visc_kind = 0;
    // learned sensor
    void* mlp_buf = nullptr;                    // w1, w2, w3 (bf16), b1, b2, b3 (f32), fallback counter
    void* powtab_buf = nullptr;                 // the power law's tables (double, then float)
    MlpArgs mlp{};
    bool mlp_on = false;
    int mlp_impl = 1;                 // learned sensor's classifier: 0 mma.sync per warp, 1 tcgen05 per CTA
    bool mlp_tuned = false;           // ensembles: classifier timed (or fixed by cfd_set_sweep_variant)
    int mlp_tc_grid = 0;              // persistent grid of the ensemble's tcgen05 walk
    bool tuned = false;
    // ensemble of blocks (cfd_create_batch): one single-block context per block
    // plus the tables that drive one persistent launch per kernel kind
    std::vector<cfd_ctx*> sub;
    SweepArgs* d_tbl[3] = {nullptr, nullptr, nullptr};  // per stage, [nb]
    int* d_maps = nullptr;                              // all prefix / gdim arrays
    BatchMap maps[3][MAP_COUNT];        // [stage][kernel kind and variant]
    int map_grid[MAP_COUNT] = {};       // persistent grid per map
    int bvar[4] = {0, 0, 0, 0};                         // chosen variant per kind (viscous, xi, eta, zeta)
    bool batch_p8 = false;  // every block periodic in every direction, 8th-order viscous terms
    // multi-block halo links: [0] between the U arrays, [1] between the Uk
    // arrays; per direction
    HaloLink* d_halo[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int n_halo[3] = {0, 0, 0};
    int* err = nullptr;             // device non-physical flag
    double* dt = nullptr;           // device scalars
    double* t = nullptr;
    unsigned long long* cflmax = nullptr;
    double* inflow = nullptr;
    double* wall_x = nullptr;
    double* wall_z = nullptr;
    double* h_pinned = nullptr;     // [8] pinned host staging: 0 err, 2 get_time, 3 set_time, 4 cfl
    bool forced = false;
    cudaGraphExec_t gexec = nullptr;
    bool graph_valid = false;
    long long launches = 0;
    int seg_len = 128;
    int bx = 128;
    size_t real_size = 8;
    std::string msg;
};

static std::string g_static_msg = "no error";

template <class R, int DIR, int EP>
static cudaError_t set_sweep_attrs();

static cfd_status fail(cfd_ctx* c, cfd_status s, const std::string& m)
{
    if (c) c->msg = m;
    else g_static_msg = m;
    return s;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, CFD_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_));        \
    } while (0)

#define LAUNCH_CHECK()                                                                            \
    do {                                                                                          \
        ++ctx->launches;                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess) return fail(ctx, CFD_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// tensor-memory-accelerator descriptors (cuTensorMapEncodeTiled, fetched
// through the runtime so that the library does not link the driver library)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// a [fields][nz][ny][nx] (rank 4) or [nz][ny][nx] (rank 3) tensor, box of
// 32 x 1 x 1 (x nbox fields)
static bool encode_rows(CUtensorMap* m, CUtensorMapDataType type, size_t esize, const void* ptr, const Geo& g,
                        int nfields, int nbox)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn || !ptr) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)nfields};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * esize, (cuuint64_t)g.nx * g.ny * esize,
                                   (cuuint64_t)g.N * esize};
    const cuuint32_t box[4] = {32, 1, 1, (cuuint32_t)nbox};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint32_t rank = nfields > 0 ? 4 : 3;
    return fn(m, type, rank, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// descriptors of the rows the TMA-staged walking sweep fetches; false when the
// grid does not meet the copy rules (rows of 32 nodes, 16-byte strides)
static bool make_row_maps(const SweepArgs& A, TmaRowMaps* m)
{
    const Geo& g = A.g;
    if (g.nx % 32 != 0) return false;
    if (!encode_rows(&m->p4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A.P, g, 7, 4)) return false;
    if (!encode_rows(&m->p1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A.P, g, 7, 1)) return false;
    if (A.Fv && !encode_rows(&m->fv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A.Fv, g, 12, 4)) return false;
    if (A.cls && !encode_rows(&m->cls, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, A.cls, g, 0, 1)) return false;
    return true;
}

static int grid_for(long long n, int block)
{
    long long b = (n + block - 1) / block;
    long long cap = (long long)kSMs * 16;
    return (int)std::max(1LL, std::min(b, cap));
}

// launch shape of the node-parallel kernels: x-chunks by ny by nz
struct NodeLaunch {
    dim3 grid, block;
};
static NodeLaunch node_launch(const Geo& g)
{
    const int bx = g.nx >= 128 ? 128 : (g.nx >= 64 ? 64 : 32);
    return {dim3((g.nx + bx - 1) / bx, g.ny, g.nz), dim3(bx)};
}

static void fill_float_consts(Phys& ph)
{
    ph.gm1f = (float)ph.gm1;
    ph.inv_gm1f = (float)ph.inv_gm1;
    ph.inv2gf = (float)ph.inv2g;
    ph.invRef = (float)ph.invRe;
    ph.kcoeff = (float)ph.kcoef;
    ph.omegaf = (float)ph.omega;
    ph.suth_sf = (float)ph.suth_s;
    ph.th1f = (float)ph.th1;
    ph.th2f = (float)ph.th2;
    ph.epsf = (float)ph.eps;
    ph.gMa2f = (float)ph.gMa2;
    ph.invMaf = (float)(1.0 / ph.Ma);
    ph.gammaf = (float)ph.gamma;
}

extern "C" void cfd_default_params(cfd_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->gamma = 1.4;
    p->Re = 0.0;
    p->Ma = 0.5;
    p->Pr = 0.72;
    p->T_wall = 1.0;
    p->T_ref = 288.15;
    p->visc_law = CFD_POWER;
    p->visc_omega = 0.76;
    p->scheme = CFD_HYBRID;
    p->theta1 = 0.02;
    p->theta2 = 0.1;
    p->visc_order = 8;
    p->metric_mode = CFD_METRIC_NODAL;
    p->precision = CFD_FP64;
    p->sensor = CFD_SENSOR_PLAIN;
    p->weno_eps = 1e-6;
}

static cfd_status validate(cfd_ctx* ctx, const cfd_grid* gr, const cfd_params* p)
{
    const int n[3] = {gr->nx, gr->ny, gr->nz};
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 1) return fail(ctx, CFD_EINVAL, "grid dimension < 1");
        for (int side = 0; side < 2; ++side) {
            int t = side ? gr->bc_hi[d] : gr->bc_lo[d];
            if (t < 0 || t > 5) return fail(ctx, CFD_EINVAL, "unknown boundary condition");
        }
        bool plo = gr->bc_lo[d] == CFD_BC_PERIODIC, phi = gr->bc_hi[d] == CFD_BC_PERIODIC;
        if (plo != phi) return fail(ctx, CFD_EINVAL, "periodic must be set on both faces of a direction");
        if (!plo && n[d] < 8) return fail(ctx, CFD_EINVAL, "non-periodic directions need >= 8 nodes");
        if ((gr->bc_lo[d] == CFD_BC_HALO || gr->bc_hi[d] == CFD_BC_HALO) && n[d] < 2 * CFD_HALO_WIDTH + 1)
            return fail(ctx, CFD_EINVAL, "a direction with ghost layers needs >= 2 CFD_HALO_WIDTH + 1 nodes");
        if (gr->bc_lo[d] == CFD_BC_INFLOW && d != 0) return fail(ctx, CFD_EINVAL, "inflow only on the xi-low face");
        if (gr->bc_hi[d] == CFD_BC_INFLOW) return fail(ctx, CFD_EINVAL, "inflow only on the xi-low face");
    }
    if (gr->ny > 65535 || gr->nz > 65535) return fail(ctx, CFD_EINVAL, "ny, nz must be <= 65535");
    if ((long long)gr->nx * gr->ny >= (1LL << 31)) return fail(ctx, CFD_EINVAL, "nx * ny must be < 2^31");
    if (gr->metric_layout < 0 || gr->metric_layout > 2) return fail(ctx, CFD_EINVAL, "bad metric_layout");
    if (!(p->gamma > 1.0) || !(p->Ma > 0.0)) return fail(ctx, CFD_EINVAL, "gamma must be > 1 and Ma > 0");
    if (p->Re > 0.0 && !(p->Pr > 0.0)) return fail(ctx, CFD_EINVAL, "Pr must be > 0");
    if (p->scheme < 0 || p->scheme > 3) return fail(ctx, CFD_EINVAL, "unknown scheme");
    if (p->recon_vars != CFD_RECON_COMPONENT && p->recon_vars != CFD_RECON_CHARACTERISTIC)
        return fail(ctx, CFD_EINVAL, "unknown recon_vars");
    if (p->visc_order != 6 && p->visc_order != 8) return fail(ctx, CFD_EINVAL, "visc_order must be 6 or 8");
    if (p->visc_law != CFD_SUTHERLAND && p->visc_law != CFD_POWER) return fail(ctx, CFD_EINVAL, "bad visc_law");
    if (p->visc_law == CFD_SUTHERLAND && !(p->T_ref > 0.0)) return fail(ctx, CFD_EINVAL, "T_ref must be > 0");
    if (!(p->weno_eps > 0.0)) return fail(ctx, CFD_EINVAL, "weno_eps must be > 0");
    if (p->metric_mode != CFD_METRIC_NODAL && p->metric_mode != CFD_METRIC_FSP)
        return fail(ctx, CFD_EINVAL, "unknown metric mode");
    if (p->metric_mode == CFD_METRIC_FSP) {
        for (int d = 0; d < 3; ++d)
            if (gr->bc_lo[d] != CFD_BC_PERIODIC)
                return fail(ctx, CFD_EUNSUPPORTED, "the free-stream-preserving metric mode needs periodic lines");
        if (p->recon_vars != CFD_RECON_COMPONENT)
            return fail(ctx, CFD_EUNSUPPORTED, "the free-stream-preserving metric mode reconstructs component-wise");
    }
    if (p->precision != CFD_FP64 && p->precision != CFD_FP32_BULK) return fail(ctx, CFD_EINVAL, "unknown precision");
    if (p->sensor != CFD_SENSOR_PLAIN && p->sensor != CFD_SENSOR_MLP) return fail(ctx, CFD_EINVAL, "unknown sensor");
    if (p->scheme == CFD_HYBRID && !(p->theta1 <= p->theta2)) return fail(ctx, CFD_EINVAL, "theta1 > theta2");
    bool wall = false;
    for (int d = 0; d < 3; ++d) wall |= gr->bc_lo[d] == CFD_BC_WALL_ISOTHERMAL || gr->bc_hi[d] == CFD_BC_WALL_ISOTHERMAL;
    if (wall && !(p->T_wall > 0.0)) return fail(ctx, CFD_EINVAL, "T_wall must be > 0");
    return CFD_OK;
}

static void free_all(cfd_ctx* c)
{
    for (cfd_ctx* b : c->sub) {
        free_all(b);
        delete b;
    }
    c->sub.clear();
    for (int s = 0; s < 3; ++s)
        if (c->d_tbl[s]) cudaFree(c->d_tbl[s]);
    for (int a = 0; a < 2; ++a)
        for (int d = 0; d < 3; ++d)
            if (c->d_halo[a][d]) cudaFree(c->d_halo[a][d]);
    if (c->d_maps) cudaFree(c->d_maps);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    void* ptrs[] = {c->b.U, c->b.Uk, c->b.P, c->b.Fv, c->b.R, c->b.cls, c->b.cls_tune, c->met, c->metf, c->err, c->dt, c->t,
                    c->mlp_buf, c->powtab_buf,
                    c->cflmax, c->inflow, c->wall_x, c->wall_z};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Host side of the table-driven power law (power_law in the kernels): for
// m_k = 1 + k/256, m_k^omega and 1/m_k; 2^(e omega) for e = -64 .. 63; the
// binomial coefficients C(omega, j), j = 1..6 (FP64) and 1..3 (FP32).  The
// table entries are evaluated in long double and rounded once.
static void power_tables(double omega, std::vector<double>& td, std::vector<float>& tf, double pc[6],
                         float pcf[3])
{
    td.assign(PT_COUNT, 0.0);
    tf.assign(PT_COUNT, 0.0f);
    const long double w = omega;
    for (int k = 0; k < 256; ++k) {
        const long double mk = 1.0L + (long double)k / 256.0L;
        td[PT_M + k] = (double)powl(mk, w);
        td[PT_INV + k] = 1.0 / (double)mk;
        tf[PT_M + k] = (float)powl(mk, w);
        tf[PT_INV + k] = (float)(1.0L / mk);
    }
    for (int e = -64; e < 64; ++e) {
        td[PT_E + e + 64] = (double)exp2l((long double)e * w);
        tf[PT_E + e + 64] = (float)exp2l((long double)e * w);
    }
    long double c = 1.0L;
    for (int j = 1; j <= 6; ++j) {
        c *= (w - (long double)(j - 1)) / (long double)j;
        pc[j - 1] = (double)c;
        if (j <= 3) pcf[j - 1] = (float)c;
    }
}

static cfd_status build_power_tables(cfd_ctx* ctx)
{
    std::vector<double> td;
    std::vector<float> tf;
    power_tables(ctx->ph.omega, td, tf, ctx->ph.pc, ctx->ph.pcf);
    const size_t bd = td.size() * sizeof(double), bf = tf.size() * sizeof(float);
    CU(cudaMalloc(&ctx->powtab_buf, bd + bf));
    CU(cudaMemcpyAsync(ctx->powtab_buf, td.data(), bd, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync((char*)ctx->powtab_buf + bd, tf.data(), bf, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->ph.powtab = (const double*)ctx->powtab_buf;
    ctx->ph.powtabf = (const float*)((char*)ctx->powtab_buf + bd);
    return CFD_OK;
}

// 1 when the metrics are one uniform diagonal matrix (a Cartesian box): the
// kernels then skip the zero off-diagonal terms (same results)
static int diagonal_metrics(int layout, const double* metrics, int on_device)
{
    if (layout != CFD_METRICS_UNIFORM) return 0;
    double m[10];
    if (on_device) {
        if (cudaMemcpy(m, metrics, sizeof(m), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    } else {
        std::memcpy(m, metrics, sizeof(m));
    }
    return m[1] == 0.0 && m[2] == 0.0 && m[3] == 0.0 && m[5] == 0.0 && m[6] == 0.0 && m[7] == 0.0;
}

// On a uniform diagonal box, the central coefficients of the viscous order
// times the metric d_x of each periodic direction (Geo::gfold, gsc)
static void fold_metrics(Geo& g, int vorder, const double* metrics, int on_device)
{
    for (int d = 0; d < 3; ++d) g.gfold[d] = 0;
    if (!g.diag) return;
    double m[10];
    if (on_device) {
        if (cudaMemcpy(m, metrics, sizeof(m), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    } else {
        std::memcpy(m, metrics, sizeof(m));
    }
    const double c8[4] = {672.0 / 840.0, -168.0 / 840.0, 32.0 / 840.0, -3.0 / 840.0};
    const double c6[4] = {45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0, 0.0};
    const double* c = vorder == 8 ? c8 : c6;
    for (int d = 0; d < 3; ++d) {
        if (!g.per[d]) continue;
        g.gfold[d] = 1;
        const double md = m[4 * d];
        for (int k = 0; k < 4; ++k) g.gsc[d][k] = c[k] * md;
    }
}

static cfd_status create_inner(cfd_ctx* ctx, const cfd_grid* grid, const double* metrics, int metrics_on_device,
                               const cfd_params* params, void* stream)
{
    ctx->grid = *grid;
    ctx->prm = *params;
    CU(cudaGetDevice(&ctx->dev));
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        CU(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    Geo& g = ctx->g;
    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.N = (long long)g.nx * g.ny * g.nz;
    for (int d = 0; d < 3; ++d) {
        g.per[d] = grid->bc_lo[d] == CFD_BC_PERIODIC;
        g.bc_lo[d] = grid->bc_lo[d];
        g.bc_hi[d] = grid->bc_hi[d];
    }
    g.mlayout = grid->metric_layout;
    g.M = g.mlayout == CFD_METRICS_3D ? g.N : (g.mlayout == CFD_METRICS_2D ? (long long)g.nx * g.ny : 1);
    g.diag = diagonal_metrics(g.mlayout, metrics, metrics_on_device);
    Phys& ph = ctx->ph;
    const cfd_params& p = *params;
    ph.gamma = p.gamma;
    ph.gm1 = p.gamma - 1.0;
    ph.inv_gm1 = 1.0 / (p.gamma - 1.0);
    ph.Ma = p.Ma;
    ph.gMa2 = p.gamma * p.Ma * p.Ma;
    ph.inv2g = 1.0 / (2.0 * p.gamma);
    ph.invMa = 1.0 / p.Ma;
    ph.viscous = p.Re > 0.0;
    ph.invRe = p.Re > 0.0 ? 1.0 / p.Re : 0.0;
    ph.kcoef = p.Re > 0.0 ? 1.0 / ((p.gamma - 1.0) * p.Ma * p.Ma * p.Pr * p.Re) : 0.0;
    ph.Tw = p.T_wall;
    ph.visc_law = p.visc_law;
    ph.omega = p.visc_omega;
    ph.suth_s = p.visc_law == CFD_SUTHERLAND ? 110.4 / p.T_ref : 0.0;
    ph.scheme = p.scheme;
    ph.charrec = p.recon_vars == CFD_RECON_CHARACTERISTIC;
    ph.th1 = p.theta1;
    ph.th2 = p.theta2;
    ph.eps = p.weno_eps;
    ph.vorder = p.visc_order;
    fill_float_consts(ph);
    fold_metrics(g, ph.vorder, metrics, metrics_on_device);
    if (ph.viscous && ph.visc_law == CFD_POWER) {
        const cfd_status sp = build_power_tables(ctx);
        if (sp != CFD_OK) return sp;
    }
    ctx->real_size = p.precision == CFD_FP32_BULK ? sizeof(float) : sizeof(double);

    const long long N = g.N;
    size_t rs = ctx->real_size;
    if (cudaMalloc(&ctx->b.U, 5 * N * sizeof(double)) != cudaSuccess) return fail(ctx, CFD_ENOMEM, "device allocation");
    CU(cudaMalloc(&ctx->b.Uk, 5 * N * sizeof(double)));
    CU(cudaMalloc(&ctx->b.P, 7 * N * rs));
    CU(cudaMalloc(&ctx->b.R, 5 * N * rs));
    CU(cudaMalloc(&ctx->b.cls, N));
    CU(cudaMemsetAsync(ctx->b.cls, 0, N, ctx->stream));
    CU(cudaMalloc(&ctx->b.cls_tune, N));
    if (ph.viscous) CU(cudaMalloc(&ctx->b.Fv, 12 * N * rs));
    CU(cudaMalloc(&ctx->met, (size_t)M_COUNT * g.M * sizeof(double)));
    CU(cudaMalloc(&ctx->err, sizeof(int)));
    CU(cudaMalloc(&ctx->dt, sizeof(double)));
    CU(cudaMalloc(&ctx->t, sizeof(double)));
    CU(cudaMalloc(&ctx->cflmax, sizeof(unsigned long long)));
    CU(cudaMallocHost(&ctx->h_pinned, 8 * sizeof(double)));
    CU(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
    CU(cudaMemsetAsync(ctx->t, 0, sizeof(double), ctx->stream));
    CU(cudaMemcpyAsync(ctx->met, metrics, 10 * g.M * sizeof(double),
                       metrics_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    g.met = ctx->met;
    k_metric_derive<<<grid_for(g.M, 256), 256, 0, ctx->stream>>>(ctx->met, g.M);
    LAUNCH_CHECK();
    CU(cudaMalloc(&ctx->metf, (size_t)M_COUNT * g.M * sizeof(float)));
    k_metric_float<<<grid_for((long long)M_COUNT * g.M, 256), 256, 0, ctx->stream>>>(ctx->met, ctx->metf,
                                                                                     (long long)M_COUNT * g.M);
    LAUNCH_CHECK();
    g.metf = ctx->metf;
    CU((set_sweep_attrs<double, 1, EP_ACCUM>()));
    CU((set_sweep_attrs<double, 2, EP_FINAL_RHS>()));
    CU((set_sweep_attrs<double, 2, EP_FINAL_RK>()));
    CU((set_sweep_attrs<float, 1, EP_ACCUM>()));
    CU((set_sweep_attrs<float, 2, EP_FINAL_RHS>()));
    CU((set_sweep_attrs<float, 2, EP_FINAL_RK>()));
    CU(cudaFuncSetAttribute(k_visc_flux25<float, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)visc25_smem_bytes<float>()));
    CU(cudaFuncSetAttribute(k_visc_flux25<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)visc25_smem_bytes<float>()));
    CU(cudaFuncSetAttribute(k_visc_flux25<double, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)visc25_smem_bytes<double>()));
    CU(cudaFuncSetAttribute(k_visc_flux25<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)visc25_smem_bytes<double>()));
    if (p.precision == CFD_FP32_BULK) CU(cudaMemsetAsync(ctx->b.cls, 2, N, ctx->stream));
    ctx->bx = g.nx <= 32 ? 32 : (g.nx <= 64 ? 64 : 128);
    CU(cudaStreamSynchronize(ctx->stream));
    return CFD_OK;
}

extern "C" cfd_status cfd_create(cfd_ctx** out, const cfd_grid* grid, const double* metrics, int metrics_on_device,
                                 const cfd_params* params, void* stream)
{
    if (!out || !grid || !metrics || !params) return fail(nullptr, CFD_EINVAL, "null argument to cfd_create");
    *out = nullptr;
    cfd_status st = validate(nullptr, grid, params);
    if (st != CFD_OK) return st;
    cfd_ctx* ctx = new (std::nothrow) cfd_ctx();
    if (!ctx) return fail(nullptr, CFD_ENOMEM, "host allocation");
    st = create_inner(ctx, grid, metrics, metrics_on_device, params, stream);
    if (st != CFD_OK) {
        g_static_msg = ctx->msg;
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        free_all(ctx);
        delete ctx;
        return st;
    }
    *out = ctx;
    return CFD_OK;
}

extern "C" void cfd_destroy(cfd_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

extern "C" const char* cfd_last_error(const cfd_ctx* ctx) { return ctx ? ctx->msg.c_str() : g_static_msg.c_str(); }

extern "C" long long cfd_launch_count(const cfd_ctx* ctx) { return ctx ? ctx->launches : 0; }

static cfd_status check_block(cfd_ctx* ctx, int block)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    const int nb = ctx->sub.empty() ? 1 : (int)ctx->sub.size();
    if (block < 0 || block >= nb) return fail(ctx, CFD_EINVAL, "block index out of range");
    return CFD_OK;
}

// run a per-block call on the block's context and copy its error message up
#define DELEGATE(call_on_sub)                                                                         \
    do {                                                                                              \
        if (!ctx->sub.empty()) {                                                                      \
            cfd_ctx* b_ = ctx->sub[block];                                                            \
            cfd_status s_ = call_on_sub;                                                              \
            if (s_ != CFD_OK) ctx->msg = b_->msg;                                                     \
            return s_;                                                                                \
        }                                                                                             \
    } while (0)

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
static bool has_nonreflect(const Geo& g)
{
    for (int d = 0; d < 3; ++d)
        if (g.bc_lo[d] == CFD_BC_NONREFLECT || g.bc_hi[d] == CFD_BC_NONREFLECT) return true;
    return false;
}

// boundary nodes through the stage's RK combination (L = 0) before the
// boundary conditions; only needed where a face is non-reflecting
static cfd_status launch_bnd_rk(cfd_ctx* ctx, const Geo& g, double* U, const double* Uin, const double* Un, double a,
                                double b)
{
    if (!Uin || !has_nonreflect(g)) return CFD_OK;
    for (int d = 0; d < 3; ++d) {
        if (g.per[d]) continue;
        long long nface = d == 0 ? (long long)g.ny * g.nz : (d == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny);
        k_bnd_rk<<<grid_for(2 * nface, 256), 256, 0, ctx->stream>>>(g, U, Uin, Un, a, b, d);
        LAUNCH_CHECK();
    }
    return CFD_OK;
}

static cfd_status launch_bc(cfd_ctx* ctx, double* U, double tfrac, bool use_dt, const double* Uin = nullptr,
                            const double* Un = nullptr, double a = 0.0, double b = 1.0)
{
    const Geo& g = ctx->g;
    {
        cfd_status sr = launch_bnd_rk(ctx, g, U, Uin, Un, a, b);
        if (sr != CFD_OK) return sr;
    }
    for (int d = 0; d < 3; ++d) {
        if (g.per[d]) continue;
        long long nface = d == 0 ? (long long)g.ny * g.nz : (d == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny);
        k_bc<<<grid_for(2 * nface, 256), 256, 0, ctx->stream>>>(g, ctx->ph, ctx->bc, U, d, ctx->t,
                                                                  use_dt ? ctx->dt : nullptr, tfrac);
        LAUNCH_CHECK();
    }
    return CFD_OK;
}

// the FP32 plain sensor rides in the node-flux kernels (kinds 0 and 3) of a
// viscous hybrid stage instead of a launch of its own
static bool sensor_fusable(const cfd_ctx* ctx)
{
    return ctx->prm.precision == CFD_FP32_BULK && ctx->ph.viscous && !ctx->forced &&
           ctx->prm.sensor == CFD_SENSOR_PLAIN;
}
static bool sensor_fused(const cfd_ctx* ctx, int visc_kind)
{
    return sensor_fusable(ctx) && (visc_kind == 0 || visc_kind == 3);
}

template <class R, bool SENS>
static void launch_visc_node(cfd_ctx* ctx, const SweepArgs& A, int kind, bool p8)
{
    const Geo& g = ctx->g;
    if (kind == 0) {
        const NodeLaunch nl = node_launch(g);
        if (p8) k_visc_flux<R, 0, true, SENS><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
        else k_visc_flux<R, 0, false, SENS><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    } else {
        dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
        if (p8) k_visc_flux<R, 4, true, SENS><<<grid, dim3(32, 4), 0, ctx->stream>>>(A);
        else k_visc_flux<R, 4, false, SENS><<<grid, dim3(32, 4), 0, ctx->stream>>>(A);
    }
}

// sens: the node-flux kernels (kinds 0, 3) also write the plain sensor's
// classes (FP32 bulk only)
template <class R>
static cfd_status launch_visc(cfd_ctx* ctx, const SweepArgs& A, int kind, bool sens = false)
{
    const Geo& g = ctx->g;
    // a periodic box with 8th-order viscous terms takes the instantiation
    // without order and closure decisions
    const bool p8 = g.per[0] && g.per[1] && g.per[2] && ctx->ph.vorder == 8;
    if (kind == 0 || kind == 3) {
        if constexpr (sizeof(R) == sizeof(float)) {
            if (sens) launch_visc_node<R, true>(ctx, A, kind, p8);
            else launch_visc_node<R, false>(ctx, A, kind, p8);
        } else {
            launch_visc_node<R, false>(ctx, A, kind, p8);
        }
    } else {
        const int tz = kind == 1 ? 64 : 32;
        dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + tz - 1) / tz);
        if (kind == 1)
            k_visc_flux25<R, 64><<<grid, 256, visc25_smem_bytes<R>(), ctx->stream>>>(A);
        else
            k_visc_flux25<R, 32><<<grid, 256, visc25_smem_bytes<R>(), ctx->stream>>>(A);
    }
    LAUNCH_CHECK();
    return CFD_OK;
}

template <class R, int DIR, int EP>
static cfd_status launch_sweep_dir(cfd_ctx* ctx, SweepArgs& A, int kind, int param)
{
    const Geo& g = ctx->g;
    const int n = DIR == 1 ? g.ny : g.nz, nother = DIR == 1 ? g.nz : g.ny;
    const int lo = g.per[DIR] ? 0 : 1, hi = g.per[DIR] ? n : n - 1;
    if (ctx->ph.charrec) {
        // characteristic reconstruction: 16-node tiles only
        dim3 grid((g.nx + 31) / 32, nother, (hi - lo + 15) / 16);
        k_sweep_t<R, DIR, EP, 16, true><<<grid, 256, tile_smem_bytes<R, 16>(), ctx->stream>>>(A);
    } else if (kind == 0) {
        A.seg_len = param;
        const long long nseg = (hi - lo + param - 1) / param;
        const long long warps = (long long)((g.nx + 31) / 32) * nother * nseg;
        k_sweep_s<R, DIR, EP><<<(unsigned)((warps + 3) / 4), 128, stream_smem_bytes<R>(), ctx->stream>>>(A);
    } else if (kind == 2 || kind == 3) {
        const int seg = param > 0 ? param : std::max(1, hi - lo);
        A.seg_len = seg;
        dim3 grid((g.nx + 31) / 32, nother, (hi - lo + seg - 1) / seg);
        TmaRowMaps maps;
        if (kind == 3 && sizeof(R) == 4 && make_row_maps(A, &maps))
            k_sweep_wt<DIR, EP><<<grid, 256, walk_tma_smem_bytes(), ctx->stream>>>(A, maps);
        else
            k_sweep_w<R, DIR, EP><<<grid, 256, walk_smem_bytes<R>(), ctx->stream>>>(A);
    } else {
        dim3 grid((g.nx + 31) / 32, nother, (hi - lo + param - 1) / param);
        // FP32 on a periodic line with 8th-order viscous terms: the
        // instantiation without order and closure decisions
        const bool p8 = sizeof(R) == 4 && g.per[DIR] && ctx->ph.vorder == 8;
        if (param == 16) {
            if (p8) k_sweep_t<R, DIR, EP, 16, false, true><<<grid, 256, tile_smem_bytes<R, 16>(), ctx->stream>>>(A);
            else k_sweep_t<R, DIR, EP, 16><<<grid, 256, tile_smem_bytes<R, 16>(), ctx->stream>>>(A);
        } else {
            if (p8) k_sweep_t<R, DIR, EP, 32, false, true><<<grid, 256, tile_smem_bytes<R, 32>(), ctx->stream>>>(A);
            else k_sweep_t<R, DIR, EP, 32><<<grid, 256, tile_smem_bytes<R, 32>(), ctx->stream>>>(A);
        }
    }
    LAUNCH_CHECK();
    return CFD_OK;
}

// xi sweep: kind 0 one CTA per segment of bx nodes (with its 8-node halo),
// kind 1 walking (seg nodes per CTA, 0 = the whole line)
template <class R>
static cfd_status launch_xi(cfd_ctx* ctx, SweepArgs& A, int kind, int seg)
{
    const Geo& g = ctx->g;
    int lo = g.per[0] ? 0 : 1, hi = g.per[0] ? g.nx : g.nx - 1;
    int nb = ctx->bx;
    dim3 grid((hi - lo + nb - 1) / nb, g.ny, g.nz);
    if (!ctx->ph.charrec && kind == 1) {
        const int sl = seg > 0 ? seg : std::max(1, hi - lo);
        dim3 gw((hi - lo + sl - 1) / sl, g.ny, g.nz);
        k_sweep_xw<R, EP_STORE><<<gw, XW, 0, ctx->stream>>>(A, sl);
    } else if (ctx->ph.charrec) {
        if (nb == 32) k_sweep_x<R, 32, EP_STORE, true><<<grid, 32, 0, ctx->stream>>>(A);
        else if (nb == 64) k_sweep_x<R, 64, EP_STORE, true><<<grid, 64, 0, ctx->stream>>>(A);
        else k_sweep_x<R, 128, EP_STORE, true><<<grid, 128, 0, ctx->stream>>>(A);
    } else if (sizeof(R) == 4 && g.per[0] && ctx->ph.vorder == 8) {
        // FP32 periodic lines, 8th-order viscous terms (as for the tiles)
        if (nb == 32) k_sweep_x<R, 32, EP_STORE, false, true><<<grid, 32, 0, ctx->stream>>>(A);
        else if (nb == 64) k_sweep_x<R, 64, EP_STORE, false, true><<<grid, 64, 0, ctx->stream>>>(A);
        else k_sweep_x<R, 128, EP_STORE, false, true><<<grid, 128, 0, ctx->stream>>>(A);
    } else if (nb == 32) {
        k_sweep_x<R, 32, EP_STORE><<<grid, 32, 0, ctx->stream>>>(A);
    } else if (nb == 64) {
        k_sweep_x<R, 64, EP_STORE><<<grid, 64, 0, ctx->stream>>>(A);
    } else {
        k_sweep_x<R, 128, EP_STORE><<<grid, 128, 0, ctx->stream>>>(A);
    }
    LAUNCH_CHECK();
    return CFD_OK;
}

template <class R, int EPF>
static cfd_status launch_sweeps(cfd_ctx* ctx, SweepArgs& A, cudaEvent_t* ev = nullptr)
{
    if (ctx->prm.metric_mode == CFD_METRIC_FSP) {
        // free-stream-preserving interface metrics: one thread per node and direction
        const NodeLaunch nl = node_launch(ctx->g);
        k_sweep_fsp<R, 0, EP_STORE><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
        LAUNCH_CHECK();
        if (ev) cudaEventRecord(ev[1], ctx->stream);
        k_sweep_fsp<R, 1, EP_ACCUM><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
        LAUNCH_CHECK();
        if (ev) cudaEventRecord(ev[2], ctx->stream);
        k_sweep_fsp<R, 2, EPF><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
        LAUNCH_CHECK();
        if (ev) cudaEventRecord(ev[3], ctx->stream);
        return CFD_OK;
    }
    {
        cfd_status sx = launch_xi<R>(ctx, A, ctx->xi_kind, ctx->xi_seg);
        if (sx != CFD_OK) return sx;
    }
    if (ev) cudaEventRecord(ev[1], ctx->stream);
    cfd_status st = launch_sweep_dir<R, 1, EP_ACCUM>(ctx, A, ctx->sweep_kind[1], ctx->sweep_param[1]);
    if (st != CFD_OK) return st;
    if (ev) cudaEventRecord(ev[2], ctx->stream);
    // zeta (final: L = J R, then RK or output)
    st = launch_sweep_dir<R, 2, EPF>(ctx, A, ctx->sweep_kind[2], ctx->sweep_param[2]);
    if (st != CFD_OK) return st;
    if (ev) cudaEventRecord(ev[3], ctx->stream);
    return CFD_OK;
}

template <class R, int DIR, int EP>
static cudaError_t set_sweep_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep_s<R, DIR, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stream_smem_bytes<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, 16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, 32>());
    // tiles are latency-bound: let the shared-memory carveout admit every
    // CTA the registers allow
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 32>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, 16>());
    if (sizeof(R) == 4) {
        const auto dyn = cudaFuncAttributeMaxDynamicSharedMemorySize;
        const auto carve = cudaFuncAttributePreferredSharedMemoryCarveout;
        const int maxs = (int)cudaSharedmemCarveoutMaxShared;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 16, false, true>, dyn,
                                                       (int)tile_smem_bytes<R, 16>());
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 32, false, true>, dyn,
                                                       (int)tile_smem_bytes<R, 32>());
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 16, false, true>, carve, maxs);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 32, false, true>, carve, maxs);
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_w<R, DIR, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)walk_smem_bytes<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_w<R, DIR, EP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && sizeof(R) == 4)
        e = cudaFuncSetAttribute(k_sweep_wt<DIR, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)walk_tma_smem_bytes());
    if (e == cudaSuccess && sizeof(R) == 4)
        e = cudaFuncSetAttribute(k_sweep_wt<DIR, EP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

static SweepArgs make_args(cfd_ctx* ctx, const double* Uin, const double* Un, double* Uout, double* Lout, double a,
                           double b)
{
    SweepArgs A{};
    A.g = ctx->g;
    A.ph = ctx->ph;
    A.P = ctx->b.P;
    A.cls = ctx->prm.scheme == CFD_HYBRID ? ctx->b.cls : nullptr;
    A.cls_io = ctx->b.cls;
    A.Fv = ctx->ph.viscous ? ctx->b.Fv : nullptr;
    A.R = ctx->b.R;
    A.err = ctx->err;
    A.U = Uin;
    A.Un = Un;
    A.Uout = Uout;
    A.Lout = Lout;
    A.dt = ctx->dt;
    A.rk_a = a;
    A.rk_b = b;
    A.seg_len = ctx->seg_len;
    return A;
}

// one evaluation of the right-hand side of Uin; EPF selects the epilogue
template <class R, int EPF>
static cfd_status run_stage_t(cfd_ctx* ctx, const double* Uin, const double* Un, double* Uout, double* Lout,
                              double a, double b, cudaEvent_t* ev)
{
    const Geo& g = ctx->g;
    const bool mixed = sizeof(R) == sizeof(float);
    SweepArgs A = make_args(ctx, Uin, Un, Uout, Lout, a, b);
    if (ev) cudaEventRecord(ev[0], ctx->stream);
    const NodeLaunch nl = node_launch(g);
    if (mixed)
        k_prim_mixed<<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    else
        k_prim<double><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[1], ctx->stream);
    const bool sensor = !ctx->forced && (mixed || ctx->prm.scheme == CFD_HYBRID);
    const bool fused = sensor && sensor_fused(ctx, ctx->visc_kind);
    const cudaStream_t sst = ctx->stream;
    if (sensor && !fused) {
        if (ctx->prm.sensor == CFD_SENSOR_MLP) {
            if (!ctx->mlp_on) return fail(ctx, CFD_EINVAL, "learned sensor selected but no weights set");
            // 32 x 8 columns walking zeta; the walk length balances the
            // waves of resident CTAs against the 7 planes each walk stages
            // before its first output
            const bool tc = ctx->mlp_impl == 1;
            const size_t smem = tc ? sizeof(MlpTcSmem) : sizeof(MlpWalkSmem);
            static int per_sm[2][2] = {{0, 0}, {0, 0}};
            int& ps = per_sm[tc][sizeof(R) == 4];
            if (!ps) {
                // (the shared-memory carveout preference first: without it the
                // occupancy query assumed one CTA per SM, and the walks were
                // sized for that)
                const auto carve = cudaFuncAttributePreferredSharedMemoryCarveout;
                const int maxs = (int)cudaSharedmemCarveoutMaxShared;
                if (tc) {
                    cudaFuncSetAttribute(k_sensor_mlp_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    cudaFuncSetAttribute(k_sensor_mlp_tc<R>, carve, maxs);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_sensor_mlp_tc<R>, 256, smem);
                } else {
                    cudaFuncSetAttribute(k_sensor_mlp<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    cudaFuncSetAttribute(k_sensor_mlp<R>, carve, maxs);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_sensor_mlp<R>, 256, smem);
                }
                ps = std::max(1, ps);
            }
            int sms = kSMs;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev);
            const long long cols = (long long)((g.nx + 31) / 32) * ((g.ny + 7) / 8);
            int tz = g.nz;
            double best = 1e300;
            for (int c : {8, 16, 32, 64}) {
                const int cz = std::min(c, g.nz);
                const long long ctas = cols * ((g.nz + cz - 1) / cz);
                const long long waves = (ctas + (long long)ps * sms - 1) / ((long long)ps * sms);
                const double cost = (double)waves * (cz + 0.3 * 7);
                if (cost < best) best = cost, tz = cz;
            }
            const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + tz - 1) / tz);
            if (tc) k_sensor_mlp_tc<R><<<grid, 256, smem, sst>>>(A, ctx->mlp, tz);
            else k_sensor_mlp<R><<<grid, 256, smem, sst>>>(A, ctx->mlp, tz);
        } else if (mixed) {
            k_sensor32<<<nl.grid, nl.block, 0, sst>>>(A);
        } else {
            k_sensor<<<nl.grid, nl.block, 0, sst>>>(A);
        }
        LAUNCH_CHECK();
    }
    if (ev) cudaEventRecord(ev[2], ctx->stream);
    if (ctx->ph.viscous) {
        cfd_status st = launch_visc<R>(ctx, A, ctx->visc_kind, fused);
        if (st != CFD_OK) return st;
    }

    if (ev) cudaEventRecord(ev[3], ctx->stream);
    return launch_sweeps<R, EPF>(ctx, A, ev ? ev + 3 : nullptr);
}

template <int EPF>
static cfd_status run_stage(cfd_ctx* ctx, const double* Uin, const double* Un, double* Uout, double* Lout,
                            double a, double b, cudaEvent_t* ev = nullptr)
{
    if (ctx->prm.precision == CFD_FP32_BULK) return run_stage_t<float, EPF>(ctx, Uin, Un, Uout, Lout, a, b, ev);
    return run_stage_t<double, EPF>(ctx, Uin, Un, Uout, Lout, a, b, ev);
}

// ---------------------------------------------------------------------------
// autotuner: picks the eta and zeta sweep variant (streaming with segment 128
// or 64, tile with 32 or 16 nodes) by timing each on the context's own state.
// Results are identical bit for bit across variants; only speed differs.
// Tuned choices are cached per process by precision, grid and scheme.
// ---------------------------------------------------------------------------
// Tuned choices are cached per process and, unless CFD_GB300_TUNE_CACHE is
// "off", in a text file (CFD_GB300_TUNE_CACHE, else
// $XDG_CACHE_HOME/paper_2209_15333_gb300/autotune.txt or
// ~/.cache/paper_2209_15333_gb300/autotune.txt), one line per entry:
//   <library build>|<GPU name>|<SMs>|<problem key>=<choice>,<choice>,...
// An entry is used only by the same library build on the same kind of GPU.
namespace {
std::mutex g_tune_mu;
bool g_tune_loaded = false;
std::vector<std::pair<std::string, std::vector<int>>> g_tune_cache;
}  // namespace

static std::string tune_file()
{
    const char* env = std::getenv("CFD_GB300_TUNE_CACHE");
    if (env && *env) return std::strcmp(env, "off") == 0 ? std::string() : std::string(env);
    std::string dir;
    if (const char* x = std::getenv("XDG_CACHE_HOME")) dir = x;
    else if (const char* h = std::getenv("HOME")) dir = std::string(h) + "/.cache";
    else return std::string();
    mkdir(dir.c_str(), 0755);
    dir += "/paper_2209_15333_gb300";
    mkdir(dir.c_str(), 0755);
    return dir + "/autotune.txt";
}

// "<build>|<GPU name>|<SMs>|" of the current device
static std::string tune_prefix(int dev)
{
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return std::string();
    }
    return std::string(__DATE__ " " __TIME__) + "|" + prop.name + "|" + std::to_string(prop.multiProcessorCount) + "|";
}

// caller holds g_tune_mu
static void tune_load_file()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_file();
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        std::string ln(line);
        while (!ln.empty() && (ln.back() == '\n' || ln.back() == '\r')) ln.pop_back();
        const size_t eq = ln.rfind('=');
        if (eq == std::string::npos) continue;
        std::vector<int> vals;
        size_t pos = eq + 1;
        bool ok = true;
        while (pos <= ln.size() && ok) {
            const size_t c = ln.find(',', pos);
            const std::string tok = ln.substr(pos, c == std::string::npos ? std::string::npos : c - pos);
            char* endp = nullptr;
            const long v = std::strtol(tok.c_str(), &endp, 10);
            ok = !tok.empty() && endp && *endp == '\0';
            vals.push_back((int)v);
            if (c == std::string::npos) break;
            pos = c + 1;
        }
        if (ok) g_tune_cache.push_back({ln.substr(0, eq), vals});
    }
    std::fclose(f);
}

static bool tune_lookup(const std::string& key, size_t nvals, std::vector<int>* out)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_file();
    for (auto it = g_tune_cache.rbegin(); it != g_tune_cache.rend(); ++it)
        if (it->first == key && it->second.size() == nvals) {
            *out = it->second;
            return true;
        }
    return false;
}

static void tune_store(const std::string& key, const std::vector<int>& vals)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back({key, vals});
    const std::string path = tune_file();
    if (path.empty()) return;
    std::string line = key + "=";
    for (size_t i = 0; i < vals.size(); ++i) line += (i ? "," : "") + std::to_string(vals[i]);
    line += "\n";
    if (FILE* f = std::fopen(path.c_str(), "a")) {
        std::fputs(line.c_str(), f);
        std::fclose(f);
    }
}

static std::string tune_key(const cfd_ctx* ctx)
{
    const Geo& g = ctx->g;
    char buf[256];
    // (the sensor kind decides whether the FP32 plain sensor rides in the
    // viscous node kernels, which changes the viscous variants' costs)
    std::snprintf(buf, sizeof(buf), "single %d %d %d %d %d%d%d %d%d%d%d%d%d %d %d %d %d %d", ctx->prm.precision, g.nx,
                  g.ny, g.nz, g.per[0], g.per[1], g.per[2], g.bc_lo[0], g.bc_lo[1], g.bc_lo[2], g.bc_hi[0],
                  g.bc_hi[1], g.bc_hi[2], ctx->prm.scheme, ctx->ph.viscous, ctx->ph.charrec, g.mlayout,
                  ctx->prm.sensor);
    return tune_prefix(ctx->dev) + buf;
}

static std::string batch_tune_key(const cfd_ctx* ctx)
{
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the block grids
    for (const cfd_ctx* sb : ctx->sub) {
        const int v[9] = {sb->g.nx, sb->g.ny, sb->g.nz, sb->g.bc_lo[0], sb->g.bc_lo[1], sb->g.bc_lo[2],
                          sb->g.bc_hi[0], sb->g.bc_hi[1], sb->g.bc_hi[2]};
        for (int x : v) {
            h ^= (unsigned long long)(unsigned)x;
            h *= 1099511628211ull;
        }
    }
    char buf[160];
    std::snprintf(buf, sizeof(buf), "batch %d %d %d %d %d %llx", ctx->prm.precision, (int)ctx->sub.size(),
                  ctx->prm.scheme, (int)ctx->ph.viscous, ctx->prm.sensor, h);
    return tune_prefix(ctx->dev) + buf;
}

// the TMA-staged walking sweep can run on this context (FP32 bulk, rows of 32
// nodes, descriptors encodable)
static bool tma_eligible(cfd_ctx* ctx)
{
    if (ctx->prm.precision != CFD_FP32_BULK || !ctx->sub.empty()) return false;
    TmaRowMaps maps;
    return make_row_maps(make_args(ctx, ctx->b.U, nullptr, nullptr, nullptr, 0.0, 1.0), &maps);
}

template <class R>
static cfd_status autotune_t(cfd_ctx* ctx)
{
    cfd_status st = run_stage<EP_FINAL_RHS>(ctx, ctx->b.U, nullptr, nullptr, ctx->b.Uk, 0.0, 1.0);
    if (st != CFD_OK) return st;
    SweepArgs A = make_args(ctx, ctx->b.U, nullptr, nullptr, ctx->b.Uk, 0.0, 1.0);
    const int cands[8][2] = {{0, 128}, {0, 64}, {1, 32}, {1, 16}, {2, 0}, {2, 64}, {3, 0}, {3, 64}};
    const int ncand = tma_eligible(ctx) ? 8 : 6;  // the TMA-staged walk is an FP32 kernel
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int dir = 1; dir <= 2 && st == CFD_OK; ++dir) {
        float best = 1e30f;
        for (int c = 0; c < ncand && st == CFD_OK; ++c) {
            for (int rep = 0; rep < 4 && st == CFD_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, ctx->stream);
                if (dir == 1) st = launch_sweep_dir<R, 1, EP_ACCUM>(ctx, A, cands[c][0], cands[c][1]);
                else st = launch_sweep_dir<R, 2, EP_FINAL_RHS>(ctx, A, cands[c][0], cands[c][1]);
            }
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ctx, CFD_ECUDA, "autotune timing");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == CFD_OK && ms < best) {
                best = ms;
                ctx->sweep_kind[dir] = cands[c][0];
                ctx->sweep_param[dir] = cands[c][1];
            }
        }
    }
    if (!ctx->ph.charrec) {
        // xi: the per-segment tiles, or walking whole lines / 256-node segments
        const int xc[3][2] = {{0, 0}, {1, 0}, {1, 256}};
        float best = 1e30f;
        for (int c = 0; c < 3 && st == CFD_OK; ++c) {
            for (int rep = 0; rep < 4 && st == CFD_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, ctx->stream);
                st = launch_xi<R>(ctx, A, xc[c][0], xc[c][1]);
            }
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ctx, CFD_ECUDA, "autotune timing");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == CFD_OK && ms < best) {
                best = ms;
                ctx->xi_kind = xc[c][0];
                ctx->xi_seg = xc[c][1];
            }
        }
    }
    if (ctx->ph.viscous) {
        // where the FP32 plain sensor can ride in the node-flux kernels, the
        // other variants are timed with the sensor launch they still need
        const bool fusable = sensor_fusable(ctx);
        float best = 1e30f;
        for (int kind = 0; kind < 4 && st == CFD_OK; ++kind) {
            for (int rep = 0; rep < 4 && st == CFD_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, ctx->stream);
                if (fusable && !sensor_fused(ctx, kind)) {
                    const NodeLaunch nl = node_launch(ctx->g);
                    k_sensor32<<<nl.grid, nl.block, 0, ctx->stream>>>(A);
                    LAUNCH_CHECK();
                }
                st = launch_visc<R>(ctx, A, kind, sensor_fused(ctx, kind));
            }
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ctx, CFD_ECUDA, "autotune timing");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == CFD_OK && ms < best) {
                best = ms;
                ctx->visc_kind = kind;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

static cfd_status autotune(cfd_ctx* ctx)
{
    if (ctx->tuned) return CFD_OK;
    if (ctx->prm.metric_mode == CFD_METRIC_FSP) {
        ctx->tuned = true;  // its sweeps have one form
        return CFD_OK;
    }
    const std::string key = tune_key(ctx);
    std::vector<int> v;
    if (tune_lookup(key, 7, &v) && v[0] >= 0 && v[0] <= 3 && v[2] >= 0 && v[2] <= 3 && v[4] >= 0 && v[4] <= 3 &&
        (v[0] != 3 || tma_eligible(ctx)) && (v[2] != 3 || tma_eligible(ctx))) {
        for (int d = 1; d <= 2; ++d) {
            ctx->sweep_kind[d] = v[2 * d - 2];
            ctx->sweep_param[d] = v[2 * d - 1];
        }
        ctx->visc_kind = v[4];
        ctx->xi_kind = v[5];
        ctx->xi_seg = v[6];
        ctx->tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    // trial runs work on a copy of the classes: the sensor they run must not
    // change what the next real evaluation sees (the mixed recovery reads it)
    CU(cudaMemcpyAsync(ctx->b.cls_tune, ctx->b.cls, ctx->g.N, cudaMemcpyDeviceToDevice, ctx->stream));
    std::swap(ctx->b.cls, ctx->b.cls_tune);
    cfd_status st = ctx->prm.precision == CFD_FP32_BULK ? autotune_t<float>(ctx) : autotune_t<double>(ctx);
    std::swap(ctx->b.cls, ctx->b.cls_tune);
    if (st != CFD_OK) return st;
    ctx->tuned = true;
    ctx->graph_valid = false;
    tune_store(key, {ctx->sweep_kind[1], ctx->sweep_param[1], ctx->sweep_kind[2], ctx->sweep_param[2], ctx->visc_kind,
                     ctx->xi_kind, ctx->xi_seg});
    return CFD_OK;
}

static void batch_variant_out(int dir, int var, int* kind, int* param);
static int batch_variant_in(int dir, int kind, int param);

extern "C" cfd_status cfd_set_sweep_variant(cfd_ctx* ctx, int dir, int kind, int param)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    if (dir == 4) {  // the learned sensor's classifier (not tuned; leaves the tuning alone)
        if (kind < 0 || kind > 1) return fail(ctx, CFD_EINVAL, "classifier kind must be 0 (mma.sync) or 1 (tcgen05)");
        ctx->mlp_impl = kind;
        ctx->mlp_tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    if (!ctx->sub.empty()) {
        const int var = dir >= 0 && dir <= 3 ? batch_variant_in(dir, kind, param) : -1;
        if (var < 0) return fail(ctx, CFD_EINVAL, "not an ensemble kernel variant");
        ctx->bvar[dir == 0 ? KIND_VISC : (dir == 3 ? KIND_SX : (dir == 1 ? KIND_T1 : KIND_T2))] = var;
        ctx->tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    if (dir == 0) {
        if (kind < 0 || kind > 3) return fail(ctx, CFD_EINVAL, "viscous kernel kind must be 0, 1, 2 or 3");
        ctx->visc_kind = kind;
        ctx->tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    if (dir == 3) {
        if (kind < 0 || kind > 1 || param < 0) return fail(ctx, CFD_EINVAL, "xi kind must be 0 or 1, param >= 0");
        ctx->xi_kind = kind;
        ctx->xi_seg = param;
        ctx->tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    if (dir < 1 || dir > 2 || kind < 0 || kind > 3) return fail(ctx, CFD_EINVAL, "dir must be 0, 1, 2 or 3");
    if (kind == 1 && param != 16 && param != 32) return fail(ctx, CFD_EINVAL, "tile length must be 16 or 32");
    if (kind == 0 && (param < 1 || param > 65535)) return fail(ctx, CFD_EINVAL, "segment length out of range");
    if (kind >= 2 && (param < 0 || param > 65535)) return fail(ctx, CFD_EINVAL, "segment length out of range");
    if (kind == 3 && !tma_eligible(ctx))
        return fail(ctx, CFD_EUNSUPPORTED, "the TMA-staged sweep needs FP32 bulk precision and nx a multiple of 32");
    ctx->sweep_kind[dir] = kind;
    ctx->sweep_param[dir] = param;
    ctx->tuned = true;
    ctx->graph_valid = false;
    return CFD_OK;
}

extern "C" cfd_status cfd_get_sweep_variant(cfd_ctx* ctx, int dir, int* kind, int* param)
{
    if (!ctx || !kind || !param || dir < 0 || dir > 4) return fail(ctx, CFD_EINVAL, "bad argument");
    if (dir == 4) {
        *kind = ctx->mlp_impl;
        *param = 0;
        return CFD_OK;
    }
    if (!ctx->sub.empty()) {
        batch_variant_out(dir, ctx->bvar[dir == 0 ? KIND_VISC : (dir == 3 ? KIND_SX : (dir == 1 ? KIND_T1 : KIND_T2))],
                          kind, param);
        return CFD_OK;
    }
    if (dir == 3) {
        *kind = ctx->xi_kind;
        *param = ctx->xi_seg;
        return CFD_OK;
    }
    if (dir == 0) {
        *kind = ctx->visc_kind;
        *param = ctx->visc_kind == 1 ? 64 : (ctx->visc_kind == 2 ? 32 : 0);
        return CFD_OK;
    }
    *kind = ctx->sweep_kind[dir];
    *param = ctx->sweep_param[dir];
    return CFD_OK;
}

static cfd_status read_err(cfd_ctx* ctx)
{
    int h = 0;
    CU(cudaMemcpyAsync(ctx->h_pinned, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    std::memcpy(&h, ctx->h_pinned, sizeof(int));
    if (h) {
        CU(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
        if (h & 2) return fail(ctx, CFD_ECUDA, "index out of bounds (caught by the bounds-checked build)");
        if (h & 8) return fail(ctx, CFD_ECUDA, "a tensor-memory-accelerator copy did not complete in time");
        if (h & 16) return fail(ctx, CFD_ECUDA, "a tensor-core (tcgen05) layer did not complete in time");
        return fail(ctx, CFD_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN) met on the device");
    }
    return CFD_OK;
}

// ---------------------------------------------------------------------------
// public entry points
// ---------------------------------------------------------------------------
extern "C" cfd_status cfd_set_inflow(cfd_ctx* ctx, const double* prim)
{
    if (!ctx || !prim) return fail(ctx, CFD_EINVAL, "null argument");
    if (!ctx->sub.empty()) return fail(ctx, CFD_EUNSUPPORTED, "inflow profiles are per single-block context");
    const int ny = ctx->g.ny;
    if (!ctx->inflow) CU(cudaMalloc(&ctx->inflow, 5 * ny * sizeof(double)));
    CU(cudaMemcpyAsync(ctx->inflow, prim, 5 * ny * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->bc.inflow = ctx->inflow;
    ctx->graph_valid = false;
    return CFD_OK;
}

extern "C" cfd_status cfd_set_blowing(cfd_ctx* ctx, double amp, double x0, double x1, double omega, int m, double Lz,
                                      const double* wall_x, const double* wall_z)
{
    if (!ctx || !wall_x || !wall_z) return fail(ctx, CFD_EINVAL, "null argument");
    if (!ctx->sub.empty()) return fail(ctx, CFD_EUNSUPPORTED, "blowing is per single-block context");
    if (!(x1 > x0) || !(Lz > 0.0)) return fail(ctx, CFD_EINVAL, "blowing strip needs x1 > x0 and Lz > 0");
    if (!ctx->wall_x) CU(cudaMalloc(&ctx->wall_x, ctx->g.nx * sizeof(double)));
    if (!ctx->wall_z) CU(cudaMalloc(&ctx->wall_z, ctx->g.nz * sizeof(double)));
    CU(cudaMemcpyAsync(ctx->wall_x, wall_x, ctx->g.nx * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->wall_z, wall_z, ctx->g.nz * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    BCData& bc = ctx->bc;
    bc.amp = amp;
    bc.x0 = x0;
    bc.x1 = x1;
    bc.omega = omega;
    bc.m = m;
    bc.Lz = Lz;
    bc.wall_x = ctx->wall_x;
    bc.wall_z = ctx->wall_z;
    ctx->graph_valid = false;
    return CFD_OK;
}

// Copy n doubles in stream order on ctx->stream.  When the host side is
// pinned, device-mapped memory the SMs move the data themselves
// (k_copy_mapped); otherwise the copy engine does.
static cfd_status copy_state(cfd_ctx* ctx, double* dst, const double* src, long long n, cudaMemcpyKind kind)
{
    if (kind != cudaMemcpyDeviceToDevice) {
        const void* host = kind == cudaMemcpyHostToDevice ? (const void*)src : (const void*)dst;
        cudaPointerAttributes at{};
        const cudaError_t qe = cudaPointerGetAttributes(&at, host);
        if (qe != cudaSuccess) cudaGetLastError();  // not a pointer the runtime knows: pageable host memory
        const bool mapped = qe == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer;
        double* d = mapped && kind == cudaMemcpyDeviceToHost ? (double*)at.devicePointer : dst;
        const double* sp = mapped && kind == cudaMemcpyHostToDevice ? (const double*)at.devicePointer : src;
        if (mapped && ((uintptr_t)d % 16) == 0 && ((uintptr_t)sp % 16) == 0) {
            const long long n2 = n / 2;
            int dev = 0, sms = 152;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            k_copy_mapped<<<sms * 8, 256, 0, ctx->stream>>>((double2*)d, (const double2*)sp, n2, d + 2 * n2,
                                                            sp + 2 * n2, (int)(n & 1));
            LAUNCH_CHECK();
            return CFD_OK;
        }
    }
    CU(cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), kind, ctx->stream));
    return CFD_OK;
}

extern "C" cfd_status cfd_set_state(cfd_ctx* ctx, int block, const double* U, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    DELEGATE(cfd_set_state(b_, 0, U, on_device));
    if (!U) return fail(ctx, CFD_EINVAL, "null state");
    const long long N = ctx->g.N;
    st = copy_state(ctx, ctx->b.U, U, 5 * N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (st != CFD_OK) return st;
    if (ctx->prm.precision == CFD_FP32_BULK && !ctx->forced) CU(cudaMemsetAsync(ctx->b.cls, 2, N, ctx->stream));
    st = launch_bc(ctx, ctx->b.U, 0.0, false);
    if (st != CFD_OK) return st;
    if (!on_device) CU(cudaStreamSynchronize(ctx->stream));
    return CFD_OK;
}

extern "C" cfd_status cfd_get_state(cfd_ctx* ctx, int block, double* U, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    DELEGATE(cfd_get_state(b_, 0, U, on_device));
    if (!U) return fail(ctx, CFD_EINVAL, "null output");
    const long long N = ctx->g.N;
    st = copy_state(ctx, U, ctx->b.U, 5 * N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    if (st != CFD_OK) return st;
    return read_err(ctx);
}

extern "C" cfd_status cfd_rhs(cfd_ctx* ctx, int block, double* dUdt, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    DELEGATE(cfd_rhs(b_, 0, dUdt, on_device));
    if (!dUdt) return fail(ctx, CFD_EINVAL, "null output");
    const long long N = ctx->g.N;
    st = autotune(ctx);
    if (st != CFD_OK) return st;
    double* Lout = dUdt;
    if (!on_device) Lout = ctx->b.Uk;  // stage buffer is free between steps
    st = run_stage<EP_FINAL_RHS>(ctx, ctx->b.U, nullptr, nullptr, Lout, 0.0, 1.0);
    if (st != CFD_OK) return st;
    if (!on_device) CU(cudaMemcpyAsync(dUdt, Lout, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return read_err(ctx);
}


// ---------------------------------------------------------------------------
// ensembles of uneven blocks (cfd_create_batch): persistent batched launches
// ---------------------------------------------------------------------------
// Work-list maps, one per kernel kind and variant: MAP_NODE flat node runs;
// viscous fluxes 2.5-D with 32 or 64 planes per item or 32 x 4 node tiles;
// xi sweep in segments of 64 / 128 nodes or walking whole lines; eta and zeta
// sweeps in 16- / 32-node tiles or walking 64-node segments.  The autotuner
// picks one variant per kind on the live ensemble (all give the same bits).

static void batch_tiles(const Geo& g, int map, int out[3])
{
    auto cdiv = [](int a, int b) { return (a + b - 1) / b; };
    auto span = [&](int d) {
        const int n = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
        return std::max(1, g.per[d] ? n : n - 2);
    };
    if (map == MAP_MLP) {  // 32 x 8 columns walking zeta segments
        out[0] = cdiv(g.nx, 32); out[1] = cdiv(g.ny, 8); out[2] = cdiv(g.nz, kBatchMlpTZ);
        return;
    }
    const int kind = map == MAP_NODE ? -1 : (map - 1) / kBatchVariants, var = (map - 1) % kBatchVariants;
    if (kind < 0) {
        out[0] = (int)((g.N + 127) / 128); out[1] = 1; out[2] = 1;  // flat node runs
    } else if (kind == KIND_VISC) {
        if (var < 2) { out[0] = cdiv(g.nx, 32); out[1] = cdiv(g.ny, 8); out[2] = cdiv(g.nz, var == 0 ? 32 : 64); }
        else { out[0] = cdiv(g.nx, 32); out[1] = cdiv(g.ny, 4); out[2] = g.nz; }
    } else if (kind == KIND_SX) {
        out[0] = var == 2 ? 1 : cdiv(span(0), var == 0 ? 64 : 128); out[1] = g.ny; out[2] = g.nz;
    } else {
        const int d = kind == KIND_T1 ? 1 : 2;
        out[0] = cdiv(g.nx, 32); out[1] = d == 1 ? g.nz : g.ny;
        out[2] = cdiv(span(d), var == 0 ? 16 : (var == 1 ? 32 : kBatchWS));
    }
}

template <class R, bool P8>
static cudaError_t batch_kernel_attrs()
{
    const auto dyn = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const auto carve = cudaFuncAttributePreferredSharedMemoryCarveout;
    const int maxs = (int)cudaSharedmemCarveoutMaxShared;
    cudaError_t e = cudaFuncSetAttribute(kb_visc_flux25<R, 32>, dyn, (int)visc25_smem_bytes<R>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_visc_flux25<R, 64>, dyn, (int)visc25_smem_bytes<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 1, EP_ACCUM, 16, P8>, dyn, (int)tile_smem_bytes<R, 16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 2, EP_FINAL_RK, 16, P8>, dyn, (int)tile_smem_bytes<R, 16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 1, EP_ACCUM, 32, P8>, dyn, (int)tile_smem_bytes<R, 32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 2, EP_FINAL_RK, 32, P8>, dyn, (int)tile_smem_bytes<R, 32>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_w<R, 1, EP_ACCUM, P8>, dyn, (int)walk_smem_bytes<R>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_w<R, 2, EP_FINAL_RK, P8>, dyn, (int)walk_smem_bytes<R>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_t<R, 1, EP_ACCUM, 16, P8>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_t<R, 2, EP_FINAL_RK, 16, P8>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_t<R, 1, EP_ACCUM, 32, P8>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_t<R, 2, EP_FINAL_RK, 32, P8>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_w<R, 1, EP_ACCUM, P8>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep_w<R, 2, EP_FINAL_RK, P8>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sensor_mlp<R>, dyn, (int)sizeof(MlpWalkSmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sensor_mlp_tc<R>, dyn, (int)sizeof(MlpTcSmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sensor_mlp<R>, carve, maxs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sensor_mlp_tc<R>, carve, maxs);
    return e;
}

// persistent grid: every SM filled to its occupancy, never more CTAs than items
template <class K>
static int persistent_grid(K kernel, int threads, size_t smem, int items)
{
    int per_sm = 1, dev = 0, sms = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    return std::max(1, std::min(items, std::max(1, per_sm) * sms));
}

template <class R, bool P8>
static void batch_grids(cfd_ctx* ctx, const int totals[MAP_COUNT])
{
    const bool mixed = sizeof(R) == sizeof(float);
    int* mg = ctx->map_grid;
    mg[MAP_NODE] = mixed ? persistent_grid(kb_prim_mixed, 128, 0, totals[MAP_NODE])
                         : persistent_grid(kb_prim<double>, 128, 0, totals[MAP_NODE]);
    mg[MAP_VISC + 0] = persistent_grid(kb_visc_flux25<R, 32>, 256, visc25_smem_bytes<R>(), totals[MAP_VISC + 0]);
    mg[MAP_VISC + 1] = persistent_grid(kb_visc_flux25<R, 64>, 256, visc25_smem_bytes<R>(), totals[MAP_VISC + 1]);
    mg[MAP_VISC + 2] = persistent_grid(kb_visc_flux_tiles<R, P8>, 128, 0, totals[MAP_VISC + 2]);
    if constexpr (sizeof(R) == sizeof(float))
        if (sensor_fusable(ctx))
            mg[MAP_VISC + 2] = persistent_grid(kb_visc_flux_tiles<R, P8, true>, 128, 0, totals[MAP_VISC + 2]);
    mg[MAP_SX + 0] = persistent_grid(kb_sweep_x<R, 64, EP_STORE, P8>, 64, 0, totals[MAP_SX + 0]);
    mg[MAP_SX + 1] = persistent_grid(kb_sweep_x<R, 128, EP_STORE, P8>, 128, 0, totals[MAP_SX + 1]);
    mg[MAP_SX + 2] = persistent_grid(kb_sweep_xw<R, EP_STORE>, XW, 0, totals[MAP_SX + 2]);
    mg[MAP_T1 + 0] =
        persistent_grid(kb_sweep_t<R, 1, EP_ACCUM, 16, P8>, 256, tile_smem_bytes<R, 16>(), totals[MAP_T1 + 0]);
    mg[MAP_T1 + 1] =
        persistent_grid(kb_sweep_t<R, 1, EP_ACCUM, 32, P8>, 256, tile_smem_bytes<R, 32>(), totals[MAP_T1 + 1]);
    mg[MAP_T1 + 2] = persistent_grid(kb_sweep_w<R, 1, EP_ACCUM, P8>, 256, walk_smem_bytes<R>(), totals[MAP_T1 + 2]);
    mg[MAP_T2 + 0] =
        persistent_grid(kb_sweep_t<R, 2, EP_FINAL_RK, 16, P8>, 256, tile_smem_bytes<R, 16>(), totals[MAP_T2 + 0]);
    mg[MAP_T2 + 1] =
        persistent_grid(kb_sweep_t<R, 2, EP_FINAL_RK, 32, P8>, 256, tile_smem_bytes<R, 32>(), totals[MAP_T2 + 1]);
    mg[MAP_T2 + 2] = persistent_grid(kb_sweep_w<R, 2, EP_FINAL_RK, P8>, 256, walk_smem_bytes<R>(), totals[MAP_T2 + 2]);
    mg[MAP_MLP] = persistent_grid(kb_sensor_mlp<R>, 256, sizeof(MlpWalkSmem), totals[MAP_MLP]);
    ctx->mlp_tc_grid = persistent_grid(kb_sensor_mlp_tc<R>, 256, sizeof(MlpTcSmem), totals[MAP_MLP]);
}

static cfd_status create_batch_inner(cfd_ctx* ctx, int nb, const cfd_grid* grids, const double* const* metrics,
                                     int metrics_on_device, const cfd_params* params, void* stream)
{
    ctx->grid = grids[0];
    ctx->prm = params[0];
    CU(cudaGetDevice(&ctx->dev));
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        CU(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    CU(cudaMalloc(&ctx->err, sizeof(int)));
    CU(cudaMalloc(&ctx->dt, sizeof(double)));
    CU(cudaMalloc(&ctx->t, sizeof(double)));
    CU(cudaMallocHost(&ctx->h_pinned, 8 * sizeof(double)));
    CU(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
    CU(cudaMemsetAsync(ctx->t, 0, sizeof(double), ctx->stream));
    ctx->ph = Phys{};
    ctx->ph.viscous = params[0].Re > 0.0;
    // the classifier an ensemble starts with; with the learned sensor its first
    // step times both and keeps the faster (on 48 blocks of 32..128 nodes per
    // axis the persistent tcgen05 walk measured 1.54 against 0.83 ms per stage,
    // while a single 256^3 box gains from it, 0.56 against 0.62 ms)
    ctx->mlp_impl = 0;
    for (int b = 0; b < nb; ++b) {
        cfd_ctx* sb = new (std::nothrow) cfd_ctx();
        if (!sb) return fail(ctx, CFD_ENOMEM, "host allocation");
        ctx->sub.push_back(sb);
        cfd_status st = create_inner(sb, &grids[b], metrics[b], metrics_on_device, &params[b], ctx->stream);
        if (st != CFD_OK) {
            ctx->msg = "block " + std::to_string(b) + ": " + sb->msg;
            return st;
        }
        if (sb->g.N >= (1LL << 31))
            return fail(ctx, CFD_EINVAL, "block " + std::to_string(b) + ": ensemble blocks hold fewer than 2^31 nodes");
    }
    // per-stage argument tables (stage 1: Uk = U + dt L(U); 2: Uk = 3/4 U + 1/4(Uk + dt L);
    // 3: U = 1/3 U + 2/3 (Uk + dt L)), sharing the ensemble's dt
    const double ra[3] = {0.0, 0.75, 1.0 / 3.0}, rb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int s = 0; s < 3; ++s) {
        std::vector<SweepArgs> tbl(nb);
        for (int b = 0; b < nb; ++b) {
            cfd_ctx* sb = ctx->sub[b];
            const double* Uin = s == 0 ? sb->b.U : sb->b.Uk;
            double* Uout = s == 2 ? sb->b.U : sb->b.Uk;
            tbl[b] = make_args(sb, Uin, sb->b.U, Uout, nullptr, ra[s], rb[s]);
            tbl[b].dt = ctx->dt;
            tbl[b].seg_len = kBatchWS;
        }
        CU(cudaMalloc(&ctx->d_tbl[s], nb * sizeof(SweepArgs)));
        CU(cudaMemcpyAsync(ctx->d_tbl[s], tbl.data(), nb * sizeof(SweepArgs), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    // work-list maps: prefix sums of tiles and per-block tile grids per kernel kind
    const int per_kind = (nb + 1) + 3 * nb;
    std::vector<int> h((size_t)MAP_COUNT * per_kind);
    int totals[MAP_COUNT];
    for (int k = 0; k < MAP_COUNT; ++k) {
        int* pre = h.data() + (size_t)k * per_kind;
        int* gd = pre + nb + 1;
        pre[0] = 0;
        for (int b = 0; b < nb; ++b) {
            batch_tiles(ctx->sub[b]->g, k, gd + 3 * b);
            pre[b + 1] = pre[b] + gd[3 * b] * gd[3 * b + 1] * gd[3 * b + 2];
        }
        totals[k] = pre[nb];
    }
    CU(cudaMalloc(&ctx->d_maps, h.size() * sizeof(int)));
    CU(cudaMemcpyAsync(ctx->d_maps, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    for (int s = 0; s < 3; ++s)
        for (int k = 0; k < MAP_COUNT; ++k) {
            int* pre = ctx->d_maps + (size_t)k * per_kind;
            ctx->maps[s][k] = BatchMap{ctx->d_tbl[s], pre, pre + nb + 1, nb};
        }
    // every block periodic in every direction with 8th-order viscous terms:
    // the viscous tiles (both forms) and the FP32 xi and tile sweeps take the
    // instantiations without order and closure decisions, as a single block does
    bool p8 = ctx->ph.viscous && params[0].visc_order == 8;
    for (int b = 0; b < nb; ++b)
        for (int d = 0; d < 3; ++d) p8 = p8 && ctx->sub[b]->g.per[d];
    ctx->batch_p8 = p8;
    if (params[0].precision == CFD_FP32_BULK) {
        if (p8) {
            CU((batch_kernel_attrs<float, true>()));
            batch_grids<float, true>(ctx, totals);
        } else {
            CU((batch_kernel_attrs<float, false>()));
            batch_grids<float, false>(ctx, totals);
        }
    } else {
        CU((batch_kernel_attrs<double, false>()));
        batch_grids<double, false>(ctx, totals);
        // the FP64 viscous tiles take the P8 instantiation (sweeps do not)
        if (p8) ctx->map_grid[MAP_VISC + 2] = persistent_grid(kb_visc_flux_tiles<double, true>, 128, 0,
                                                              totals[MAP_VISC + 2]);
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return CFD_OK;
}

static cfd_status launch_halo(cfd_ctx* ctx, int which);

extern "C" cfd_status cfd_set_halo_links(cfd_ctx* ctx, const int* links)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    if (ctx->sub.empty()) return fail(ctx, CFD_EINVAL, "halo links join the blocks of an ensemble");
    const int nb = (int)ctx->sub.size();
    const int H = CFD_HALO_WIDTH;
    std::vector<HaloLink> h[2][3];
    if (links) {
        for (int b = 0; b < nb; ++b)
            for (int d = 0; d < 3; ++d)
                for (int side = 0; side < 2; ++side) {
                    const int c = links[(b * 3 + d) * 2 + side];
                    const Geo& gb = ctx->sub[b]->g;
                    const int tb = side ? gb.bc_hi[d] : gb.bc_lo[d];
                    if (c < 0) {
                        if (tb == CFD_BC_HALO) return fail(ctx, CFD_EINVAL, "a HALO face without a link");
                        continue;
                    }
                    if (c >= nb) return fail(ctx, CFD_EINVAL, "halo link to a block that does not exist");
                    if (tb != CFD_BC_HALO) return fail(ctx, CFD_EINVAL, "a linked face must be CFD_BC_HALO");
                    const Geo& gc = ctx->sub[c]->g;
                    const int db[3] = {gb.nx, gb.ny, gb.nz}, dc[3] = {gc.nx, gc.ny, gc.nz};
                    const int a = (d + 1) % 3, e = (d + 2) % 3;
                    if (db[a] != dc[a] || db[e] != dc[e])
                        return fail(ctx, CFD_EINVAL, "linked blocks differ across the shared face");
                    if (dc[d] < 2 * H + 1) return fail(ctx, CFD_EINVAL, "neighbour too thin for its ghost layers");
                    for (int w = 0; w < 2; ++w) {
                        HaloLink L;
                        L.dst = w ? ctx->sub[b]->b.Uk : ctx->sub[b]->b.U;
                        L.src = w ? ctx->sub[c]->b.Uk : ctx->sub[c]->b.U;
                        L.dstN = gb.N;
                        L.srcN = gc.N;
                        L.dnx = gb.nx; L.dny = gb.ny; L.snx = gc.nx; L.sny = gc.ny;
                        L.dl0 = side ? db[d] - H : 0;
                        L.sl0 = side ? H : dc[d] - 2 * H;
                        L.na = db[a];
                        L.nb = db[e];
                        h[w][d].push_back(L);
                    }
                }
    }
    for (int w = 0; w < 2; ++w)
        for (int d = 0; d < 3; ++d) {
            if (ctx->d_halo[w][d]) {
                CU(cudaStreamSynchronize(ctx->stream));
                CU(cudaFree(ctx->d_halo[w][d]));
                ctx->d_halo[w][d] = nullptr;
            }
            if (!h[w][d].empty()) {
                CU(cudaMalloc(&ctx->d_halo[w][d], h[w][d].size() * sizeof(HaloLink)));
                CU(cudaMemcpyAsync(ctx->d_halo[w][d], h[w][d].data(), h[w][d].size() * sizeof(HaloLink),
                                   cudaMemcpyHostToDevice, ctx->stream));
            }
            ctx->n_halo[d] = (int)h[0][d].size();
        }
    ctx->graph_valid = false;
    cfd_status st = launch_halo(ctx, 0);
    if (st != CFD_OK) return st;
    CU(cudaStreamSynchronize(ctx->stream));
    return CFD_OK;
}

extern "C" cfd_status cfd_create_batch(cfd_ctx** out, int nblocks, const cfd_grid* grids,
                                       const double* const* metrics, int metrics_on_device, const cfd_params* params,
                                       void* stream)
{
    if (!out || !grids || !metrics || !params || nblocks < 1)
        return fail(nullptr, CFD_EINVAL, "bad argument to cfd_create_batch");
    *out = nullptr;
    for (int b = 0; b < nblocks; ++b) {
        if (!metrics[b]) return fail(nullptr, CFD_EINVAL, "null metrics for a block");
        cfd_status st = validate(nullptr, &grids[b], &params[b]);
        if (st != CFD_OK) return st;
        const cfd_params &p = params[b], &p0 = params[0];
        if (p.precision != p0.precision || p.scheme != p0.scheme || (p.Re > 0.0) != (p0.Re > 0.0) ||
            p.visc_order != p0.visc_order || p.metric_mode != p0.metric_mode || p.sensor != p0.sensor ||
            p.recon_vars != p0.recon_vars)
            return fail(nullptr, CFD_EINVAL,
                        "all blocks of a batch share precision, scheme, viscous/inviscid, visc_order and sensor");
        if (p.recon_vars != CFD_RECON_COMPONENT)
            return fail(nullptr, CFD_EUNSUPPORTED, "characteristic reconstruction: single-block contexts only");
        if (p.metric_mode != CFD_METRIC_NODAL)
            return fail(nullptr, CFD_EUNSUPPORTED, "the free-stream-preserving mode: single-block contexts only");
    }
    cfd_ctx* ctx = new (std::nothrow) cfd_ctx();
    if (!ctx) return fail(nullptr, CFD_ENOMEM, "host allocation");
    cfd_status st = create_batch_inner(ctx, nblocks, grids, metrics, metrics_on_device, params, stream);
    if (st != CFD_OK) {
        g_static_msg = ctx->msg;
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        free_all(ctx);
        delete ctx;
        return st;
    }
    *out = ctx;
    return CFD_OK;
}

// the FP32 plain sensor rides in the ensemble's viscous node tiles (variant 2)
static bool batch_sensor_fused(const cfd_ctx* ctx, int visc_var)
{
    return sensor_fusable(ctx) && visc_var == 2;
}

// one persistent launch of kernel kind `kind` (KIND_*) in variant `var` for
// stage s of the ensemble
template <class R, bool P8>
static cfd_status launch_batch_kind_t(cfd_ctx* ctx, int s, int kind, int var)
{
    const cudaStream_t st = ctx->stream;
    const BatchMap* m = ctx->maps[s];
    const int* mg = ctx->map_grid;
    switch (kind) {
    case KIND_VISC:
        if (var == 0) kb_visc_flux25<R, 32><<<mg[MAP_VISC], 256, visc25_smem_bytes<R>(), st>>>(m[MAP_VISC]);
        else if (var == 1) kb_visc_flux25<R, 64><<<mg[MAP_VISC + 1], 256, visc25_smem_bytes<R>(), st>>>(m[MAP_VISC + 1]);
        else if (batch_sensor_fused(ctx, var)) {
            if constexpr (sizeof(R) == sizeof(float)) {
                if (ctx->batch_p8)
                    kb_visc_flux_tiles<R, true, true><<<mg[MAP_VISC + 2], dim3(32, 4), 0, st>>>(m[MAP_VISC + 2]);
                else kb_visc_flux_tiles<R, false, true><<<mg[MAP_VISC + 2], dim3(32, 4), 0, st>>>(m[MAP_VISC + 2]);
            }
        } else if (ctx->batch_p8) kb_visc_flux_tiles<R, true><<<mg[MAP_VISC + 2], dim3(32, 4), 0, st>>>(m[MAP_VISC + 2]);
        else kb_visc_flux_tiles<R><<<mg[MAP_VISC + 2], dim3(32, 4), 0, st>>>(m[MAP_VISC + 2]);
        break;
    case KIND_SX:
        if (var == 0) kb_sweep_x<R, 64, EP_STORE, P8><<<mg[MAP_SX], 64, 0, st>>>(m[MAP_SX]);
        else if (var == 1) kb_sweep_x<R, 128, EP_STORE, P8><<<mg[MAP_SX + 1], 128, 0, st>>>(m[MAP_SX + 1]);
        else kb_sweep_xw<R, EP_STORE><<<mg[MAP_SX + 2], XW, 0, st>>>(m[MAP_SX + 2]);
        break;
    case KIND_T1:
        if (var == 0)
            kb_sweep_t<R, 1, EP_ACCUM, 16, P8><<<mg[MAP_T1], 256, tile_smem_bytes<R, 16>(), st>>>(m[MAP_T1]);
        else if (var == 1)
            kb_sweep_t<R, 1, EP_ACCUM, 32, P8><<<mg[MAP_T1 + 1], 256, tile_smem_bytes<R, 32>(), st>>>(m[MAP_T1 + 1]);
        else kb_sweep_w<R, 1, EP_ACCUM, P8><<<mg[MAP_T1 + 2], 256, walk_smem_bytes<R>(), st>>>(m[MAP_T1 + 2]);
        break;
    default:
        if (var == 0)
            kb_sweep_t<R, 2, EP_FINAL_RK, 16, P8><<<mg[MAP_T2], 256, tile_smem_bytes<R, 16>(), st>>>(m[MAP_T2]);
        else if (var == 1)
            kb_sweep_t<R, 2, EP_FINAL_RK, 32, P8><<<mg[MAP_T2 + 1], 256, tile_smem_bytes<R, 32>(), st>>>(
                m[MAP_T2 + 1]);
        else kb_sweep_w<R, 2, EP_FINAL_RK, P8><<<mg[MAP_T2 + 2], 256, walk_smem_bytes<R>(), st>>>(m[MAP_T2 + 2]);
        break;
    }
    LAUNCH_CHECK();
    return CFD_OK;
}

// the sweeps take the P8 instantiations in FP32 only (as for one block)
template <class R>
static cfd_status launch_batch_kind(cfd_ctx* ctx, int s, int kind, int var)
{
    if (sizeof(R) == sizeof(float) && ctx->batch_p8) return launch_batch_kind_t<R, true>(ctx, s, kind, var);
    return launch_batch_kind_t<R, false>(ctx, s, kind, var);
}

template <class R>
static cfd_status enqueue_batch_stage(cfd_ctx* ctx, int s, cudaEvent_t* ev)
{
    const bool mixed = sizeof(R) == sizeof(float);
    const cudaStream_t st = ctx->stream;
    const BatchMap* m = ctx->maps[s];
    if (ev) cudaEventRecord(ev[0], st);
    if (mixed) kb_prim_mixed<<<ctx->map_grid[MAP_NODE], 128, 0, st>>>(m[MAP_NODE]);
    else kb_prim<double><<<ctx->map_grid[MAP_NODE], 128, 0, st>>>(m[MAP_NODE]);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[1], st);
    if (mixed || ctx->prm.scheme == CFD_HYBRID) {
        if (ctx->prm.sensor == CFD_SENSOR_MLP) {
            if (!ctx->mlp_on) return fail(ctx, CFD_EINVAL, "learned sensor selected but no weights set");
            if (ctx->mlp_impl == 1)
                kb_sensor_mlp_tc<R><<<ctx->mlp_tc_grid, 256, sizeof(MlpTcSmem), st>>>(m[MAP_MLP], ctx->mlp,
                                                                                      kBatchMlpTZ);
            else
                kb_sensor_mlp<R><<<ctx->map_grid[MAP_MLP], 256, sizeof(MlpWalkSmem), st>>>(m[MAP_MLP], ctx->mlp,
                                                                                           kBatchMlpTZ);
            LAUNCH_CHECK();
        } else if (mixed) {
            // (the viscous node tiles may form these classes instead)
            if (!batch_sensor_fused(ctx, ctx->bvar[KIND_VISC])) {
                kb_sensor32<<<ctx->map_grid[MAP_NODE], 128, 0, st>>>(m[MAP_NODE]);
                LAUNCH_CHECK();
            }
        } else {
            kb_sensor<<<ctx->map_grid[MAP_NODE], 128, 0, st>>>(m[MAP_NODE]);
            LAUNCH_CHECK();
        }
    }
    if (ev) cudaEventRecord(ev[2], st);
    if (ctx->ph.viscous) {
        cfd_status sv = launch_batch_kind<R>(ctx, s, KIND_VISC, ctx->bvar[KIND_VISC]);
        if (sv != CFD_OK) return sv;
    }
    if (ev) cudaEventRecord(ev[3], st);
    for (int kind = KIND_SX; kind <= KIND_T2; ++kind) {
        cfd_status sk = launch_batch_kind<R>(ctx, s, kind, ctx->bvar[kind]);
        if (sk != CFD_OK) return sk;
        if (ev) cudaEventRecord(ev[3 + kind], st);
    }
    // boundary conditions of blocks with non-periodic faces, at the stage time
    const double tfrac[3] = {1.0, 0.5, 1.0};
    const double ra[3] = {0.0, 0.75, 1.0 / 3.0}, rb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (cfd_ctx* sb : ctx->sub) {
        double* Uout = s == 2 ? sb->b.U : sb->b.Uk;
        {
            cfd_status sr = launch_bnd_rk(ctx, sb->g, Uout, s == 0 ? sb->b.U : sb->b.Uk, sb->b.U, ra[s], rb[s]);
            if (sr != CFD_OK) return sr;
        }
        for (int d = 0; d < 3; ++d) {
            if (sb->g.per[d]) continue;
            const Geo& g = sb->g;
            long long nface = d == 0 ? (long long)g.ny * g.nz : (d == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny);
            k_bc<<<grid_for(2 * nface, 256), 256, 0, st>>>(g, sb->ph, sb->bc, Uout, d, ctx->t, ctx->dt, tfrac[s]);
            LAUNCH_CHECK();
        }
    }
    return CFD_OK;
}

// ghost layers of linked faces from the neighbours' interiors: which = 0 the
// U arrays, 1 the Uk arrays; xi, then eta, then zeta
static cfd_status launch_halo(cfd_ctx* ctx, int which)
{
    for (int d = 0; d < 3; ++d) {
        if (!ctx->n_halo[d]) continue;
        k_halo<<<dim3(128, ctx->n_halo[d]), 256, 0, ctx->stream>>>(ctx->d_halo[which][d], d, CFD_HALO_WIDTH);
        LAUNCH_CHECK();
    }
    return CFD_OK;
}

// Ensemble autotuner: times every variant of each kernel kind on the live
// work lists of a stage-1 evaluation and keeps the fastest.  Trial runs write
// only stage buffers; the classes the mixed recovery reads next are saved and
// restored around them.
template <class R>
static cfd_status batch_autotune_t(cfd_ctx* ctx)
{
    for (cfd_ctx* sb : ctx->sub)
        CU(cudaMemcpyAsync(sb->b.cls_tune, sb->b.cls, sb->g.N, cudaMemcpyDeviceToDevice, ctx->stream));
    cfd_status st = enqueue_batch_stage<R>(ctx, 0, nullptr);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int kind = 0; kind < KIND_COUNT && st == CFD_OK; ++kind) {
        if (kind == KIND_VISC && !ctx->ph.viscous) continue;
        float best = 1e30f;
        for (int var = 0; var < kBatchVariants && st == CFD_OK; ++var) {
            for (int rep = 0; rep < 4 && st == CFD_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, ctx->stream);
                // viscous variants that leave the FP32 plain sensor to its own
                // launch are timed with it
                if (kind == KIND_VISC && sensor_fusable(ctx) && !batch_sensor_fused(ctx, var)) {
                    kb_sensor32<<<ctx->map_grid[MAP_NODE], 128, 0, ctx->stream>>>(ctx->maps[0][MAP_NODE]);
                    LAUNCH_CHECK();
                }
                st = launch_batch_kind<R>(ctx, 0, kind, var);
            }
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ctx, CFD_ECUDA, "ensemble autotune timing");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == CFD_OK && ms < best) {
                best = ms;
                ctx->bvar[kind] = var;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (cfd_ctx* sb : ctx->sub)
        CU(cudaMemcpyAsync(sb->b.cls, sb->b.cls_tune, sb->g.N, cudaMemcpyDeviceToDevice, ctx->stream));
    return st;
}

// Ensembles with the learned sensor: time both classifiers (mma.sync and
// tcgen05) once on the live work list and keep the faster.  The trial launches
// count no fallbacks, and the classes the mixed recovery reads next are saved
// and restored around them.
template <class R>
static cfd_status batch_tune_mlp_t(cfd_ctx* ctx)
{
    const cudaStream_t st = ctx->stream;
    const BatchMap* m = ctx->maps[0];
    for (cfd_ctx* sb : ctx->sub)
        CU(cudaMemcpyAsync(sb->b.cls_tune, sb->b.cls, sb->g.N, cudaMemcpyDeviceToDevice, st));
    // primitives of the state, which the features read
    if (sizeof(R) == sizeof(float)) kb_prim_mixed<<<ctx->map_grid[MAP_NODE], 128, 0, st>>>(m[MAP_NODE]);
    else kb_prim<double><<<ctx->map_grid[MAP_NODE], 128, 0, st>>>(m[MAP_NODE]);
    LAUNCH_CHECK();
    MlpArgs W = ctx->mlp;
    W.fallbacks = nullptr;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    cfd_status res = CFD_OK;
    for (int impl = 0; impl < 2 && res == CFD_OK; ++impl) {
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            if (impl == 1)
                kb_sensor_mlp_tc<R><<<ctx->mlp_tc_grid, 256, sizeof(MlpTcSmem), st>>>(m[MAP_MLP], W, kBatchMlpTZ);
            else
                kb_sensor_mlp<R><<<ctx->map_grid[MAP_MLP], 256, sizeof(MlpWalkSmem), st>>>(m[MAP_MLP], W, kBatchMlpTZ);
            ++ctx->launches;
            if (cudaGetLastError() != cudaSuccess) res = fail(ctx, CFD_ECUDA, "classifier trial launch");
        }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) res = fail(ctx, CFD_ECUDA, "classifier timing");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (res == CFD_OK && ms < best) {
            best = ms;
            ctx->mlp_impl = impl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (res != CFD_OK) return res;
    for (cfd_ctx* sb : ctx->sub)
        CU(cudaMemcpyAsync(sb->b.cls, sb->b.cls_tune, sb->g.N, cudaMemcpyDeviceToDevice, st));
    ctx->mlp_tuned = true;
    ctx->graph_valid = false;
    return read_err(ctx);
}

static cfd_status batch_autotune(cfd_ctx* ctx)
{
    if (ctx->tuned) return CFD_OK;
    const std::string key = batch_tune_key(ctx);
    std::vector<int> v;
    if (tune_lookup(key, KIND_COUNT, &v) && *std::min_element(v.begin(), v.end()) >= 0 &&
        *std::max_element(v.begin(), v.end()) < kBatchVariants) {
        for (int k = 0; k < KIND_COUNT; ++k) ctx->bvar[k] = v[k];
        ctx->tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    cfd_status st = ctx->prm.precision == CFD_FP32_BULK ? batch_autotune_t<float>(ctx) : batch_autotune_t<double>(ctx);
    if (st != CFD_OK) return st;
    ctx->tuned = true;
    ctx->graph_valid = false;
    tune_store(key, std::vector<int>(ctx->bvar, ctx->bvar + KIND_COUNT));
    return CFD_OK;
}

// ensemble variants in the (kind, param) vocabulary of cfd_set_sweep_variant
static void batch_variant_out(int dir, int var, int* kind, int* param)
{
    static const int visc[3][2] = {{2, 32}, {1, 64}, {3, 0}};
    static const int xi[3][2] = {{0, 64}, {0, 128}, {1, 0}};
    static const int eta[3][2] = {{1, 16}, {1, 32}, {2, kBatchWS}};
    const int(*t)[2] = dir == 0 ? visc : (dir == 3 ? xi : eta);
    *kind = t[var][0];
    *param = t[var][1];
}

static int batch_variant_in(int dir, int kind, int param)
{
    if (dir == 0) return kind == 2 ? 0 : (kind == 1 ? 1 : (kind == 3 ? 2 : -1));
    if (dir == 3) return kind == 1 ? 2 : (kind == 0 && param == 64 ? 0 : (kind == 0 && param == 128 ? 1 : -1));
    return kind == 2 ? 2 : (kind == 1 && param == 16 ? 0 : (kind == 1 && param == 32 ? 1 : -1));
}

static cfd_status enqueue_batch_step(cfd_ctx* ctx)
{
    for (int s = 0; s < 3; ++s) {
        // stage s reads U (s = 0) or Uk: refresh its ghost layers first
        cfd_status sh = launch_halo(ctx, s == 0 ? 0 : 1);
        if (sh != CFD_OK) return sh;
        cfd_status st = ctx->prm.precision == CFD_FP32_BULK ? enqueue_batch_stage<float>(ctx, s, nullptr)
                                                            : enqueue_batch_stage<double>(ctx, s, nullptr);
        if (st != CFD_OK) return st;
    }
    k_advance_time<<<1, 32, 0, ctx->stream>>>(ctx->t, ctx->dt);
    LAUNCH_CHECK();
    return CFD_OK;
}

static cfd_status enqueue_step(cfd_ctx* ctx)
{
    if (!ctx->sub.empty()) return enqueue_batch_step(ctx);
    cfd_status st;
    // stage 1: Uk = U + dt L(U)
    st = run_stage<EP_FINAL_RK>(ctx, ctx->b.U, ctx->b.U, ctx->b.Uk, nullptr, 0.0, 1.0);
    if (st != CFD_OK) return st;
    st = launch_bc(ctx, ctx->b.Uk, 1.0, true, ctx->b.U, ctx->b.U, 0.0, 1.0);
    if (st != CFD_OK) return st;
    // stage 2: Uk = 3/4 U + 1/4 (Uk + dt L(Uk))
    st = run_stage<EP_FINAL_RK>(ctx, ctx->b.Uk, ctx->b.U, ctx->b.Uk, nullptr, 0.75, 0.25);
    if (st != CFD_OK) return st;
    st = launch_bc(ctx, ctx->b.Uk, 0.5, true, ctx->b.Uk, ctx->b.U, 0.75, 0.25);
    if (st != CFD_OK) return st;
    // stage 3: U = 1/3 U + 2/3 (Uk + dt L(Uk))
    st = run_stage<EP_FINAL_RK>(ctx, ctx->b.Uk, ctx->b.U, ctx->b.U, nullptr, 1.0 / 3.0, 2.0 / 3.0);
    if (st != CFD_OK) return st;
    st = launch_bc(ctx, ctx->b.U, 1.0, true, ctx->b.Uk, ctx->b.U, 1.0 / 3.0, 2.0 / 3.0);
    if (st != CFD_OK) return st;
    k_advance_time<<<1, 32, 0, ctx->stream>>>(ctx->t, ctx->dt);
    LAUNCH_CHECK();
    return CFD_OK;
}

static cfd_status build_graph(cfd_ctx* ctx)
{
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    long long before = ctx->launches;
    cfd_status st = enqueue_step(ctx);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != CFD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(ctx, CFD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    ctx->launches = before;  // capture issues no work
    e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, CFD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->graph_valid = true;
    return CFD_OK;
}

static long long launches_per_step(const cfd_ctx* ctx)
{
    if (!ctx->sub.empty()) {
        const bool sensor = ctx->prm.scheme == CFD_HYBRID || ctx->prm.precision == CFD_FP32_BULK;
        long long per_stage = 1 + 3 + (sensor ? 1 : 0) + (ctx->ph.viscous ? 1 : 0);
        for (const cfd_ctx* sb : ctx->sub)
            for (int d = 0; d < 3; ++d) per_stage += sb->g.per[d] ? 0 : (has_nonreflect(sb->g) ? 2 : 1);
        return 3 * per_stage + 1;
    }
    const bool sensor = !ctx->forced && (ctx->prm.scheme == CFD_HYBRID || ctx->prm.precision == CFD_FP32_BULK);
    long long per_stage = 1 + 3 + (sensor ? 1 : 0) + (ctx->ph.viscous ? 1 : 0);
    long long bc = 0;
    for (int d = 0; d < 3; ++d) bc += ctx->g.per[d] ? 0 : (has_nonreflect(ctx->g) ? 2 : 1);
    return 3 * (per_stage + bc) + 1;
}

extern "C" cfd_status cfd_step(cfd_ctx* ctx, double dt, int nsteps)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    if (!(dt > 0.0) || nsteps < 0) return fail(ctx, CFD_EINVAL, "dt must be > 0 and nsteps >= 0");
    if (nsteps == 0) return CFD_OK;
    k_set_scalar<<<1, 32, 0, ctx->stream>>>(ctx->dt, dt);
    LAUNCH_CHECK();
    {
        cfd_status st = ctx->sub.empty() ? autotune(ctx) : batch_autotune(ctx);
        if (st != CFD_OK) return st;
        if (!ctx->sub.empty() && ctx->mlp_on && !ctx->mlp_tuned && ctx->prm.sensor == CFD_SENSOR_MLP)
            st = ctx->prm.precision == CFD_FP32_BULK ? batch_tune_mlp_t<float>(ctx) : batch_tune_mlp_t<double>(ctx);
        if (st != CFD_OK) return st;
    }
    if (!ctx->graph_valid) {
        cfd_status st = build_graph(ctx);
        if (st != CFD_OK) return st;
    }
    for (int s = 0; s < nsteps; ++s) {
        CU(cudaGraphLaunch(ctx->gexec, ctx->stream));
        ctx->launches += launches_per_step(ctx);
    }
    return CFD_OK;
}

extern "C" cfd_status cfd_cfl_dt(cfd_ctx* ctx, int block, double cfl, double* dt)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    DELEGATE(cfd_cfl_dt(b_, 0, cfl, dt));
    if (!dt || !(cfl > 0.0)) return fail(ctx, CFD_EINVAL, "bad cfl or null output");
    const Geo& g = ctx->g;
    const bool mixed = ctx->prm.precision == CFD_FP32_BULK;
    const NodeLaunch nl = node_launch(g);
    const SweepArgs A = make_args(ctx, ctx->b.U, nullptr, nullptr, nullptr, 0.0, 1.0);
    if (mixed)
        k_prim_mixed<<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    else
        k_prim<double><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    LAUNCH_CHECK();
    CU(cudaMemsetAsync(ctx->cflmax, 0, sizeof(unsigned long long), ctx->stream));
    if (mixed)
        k_cfl<float><<<grid_for(g.N, 256), 256, 0, ctx->stream>>>(g, (const float*)ctx->b.P, ctx->cflmax);
    else
        k_cfl<double><<<grid_for(g.N, 256), 256, 0, ctx->stream>>>(g, (const double*)ctx->b.P, ctx->cflmax);
    LAUNCH_CHECK();
    CU(cudaMemcpyAsync(ctx->h_pinned + 4, ctx->cflmax, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    st = read_err(ctx);
    if (st != CFD_OK) return st;
    double mx;
    std::memcpy(&mx, ctx->h_pinned + 4, sizeof(double));
    if (!(mx > 0.0)) return fail(ctx, CFD_ENONPHYS, "zero characteristic speed");
    *dt = cfl / mx;
    return CFD_OK;
}

extern "C" cfd_status cfd_get_flags(cfd_ctx* ctx, int block, unsigned char* cls, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    DELEGATE(cfd_get_flags(b_, 0, cls, on_device));
    if (!cls) return fail(ctx, CFD_EINVAL, "null output");
    CU(cudaMemcpyAsync(cls, ctx->b.cls, ctx->g.N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return CFD_OK;
}

extern "C" cfd_status cfd_force_flags(cfd_ctx* ctx, int block, const unsigned char* cls, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    if (!ctx->sub.empty()) return fail(ctx, CFD_EUNSUPPORTED, "forced classes are per single-block context");
    if (!cls) {
        ctx->forced = false;
    } else {
        CU(cudaMemcpyAsync(ctx->b.cls, cls, ctx->g.N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->forced = true;
    }
    ctx->graph_valid = false;
    return CFD_OK;
}

extern "C" cfd_status cfd_get_time(cfd_ctx* ctx, double* t)
{
    if (!ctx || !t) return fail(ctx, CFD_EINVAL, "null argument");
    CU(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->t, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *t = ctx->h_pinned[2];
    return CFD_OK;
}

extern "C" cfd_status cfd_set_time(cfd_ctx* ctx, double t)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    ctx->h_pinned[3] = t;
    CU(cudaMemcpyAsync(ctx->t, ctx->h_pinned + 3, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (cfd_ctx* b : ctx->sub) {
        cfd_status st = cfd_set_time(b, t);
        if (st != CFD_OK) return st;
    }
    return CFD_OK;
}

extern "C" cfd_status cfd_sync(cfd_ctx* ctx, double timeout_s)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return fail(ctx, CFD_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_s) return fail(ctx, CFD_ETIMEOUT, "cfd_sync timed out; work still running");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (cfd_ctx* b : ctx->sub) {
        cfd_status st = read_err(b);
        if (st != CFD_OK) {
            ctx->msg = b->msg;
            return st;
        }
    }
    return read_err(ctx);
}

extern "C" cfd_status cfd_fma_peak(int precision, double* tflops)
{
    cfd_ctx* ctx = nullptr;
    if (!tflops || (precision != CFD_FP64 && precision != CFD_FP32_BULK))
        return fail(nullptr, CFD_EINVAL, "bad argument to cfd_fma_peak");
    int dev = 0, sms = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* out = nullptr;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&out, 16);
    const int threads = 256, blocks = sms * 8;
    const int iters = precision == CFD_FP64 ? 2048 : 65536;
    float ms = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        if (precision == CFD_FP64)
            k_fma_probe<double><<<blocks, threads, 0, st>>>((double*)out, iters, 0.999999, 1e-7);
        else
            k_fma_probe<float><<<blocks, threads, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess) {
        double flops = 2.0 * 8.0 * iters * (double)threads * blocks;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(ctx, CFD_ECUDA, std::string("fma probe: ") + cudaGetErrorString(e));
    return CFD_OK;
}

extern "C" cfd_status cfd_check_conversions(unsigned long long* counts)
{
    if (!counts) return fail(nullptr, CFD_EINVAL, "bad argument to cfd_check_conversions");
    int dev = 0, sms = 0;
    cudaStream_t st = nullptr;
    unsigned long long* out = nullptr;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&out, CFD_CHECK_CONVERSIONS * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, CFD_CHECK_CONVERSIONS * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        k_check_conversions<<<sms * 8, 256, 0, st>>>(out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, out, CFD_CHECK_CONVERSIONS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (out) cudaFree(out);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(nullptr, CFD_ECUDA, std::string("conversion check: ") + cudaGetErrorString(e));
    return CFD_OK;
}

extern "C" cfd_status cfd_profile_stage(cfd_ctx* ctx, int reps, double* ms)
{
    if (!ctx || !ms || reps < 1) return fail(ctx, CFD_EINVAL, "bad argument to cfd_profile_stage");
    if (!ctx->sub.empty()) {
        // ensemble: time the persistent launches of one stage-1 evaluation
        // (it writes the stage buffers only); [3] is the xi sweep, [4] eta, [5] zeta
        cudaEvent_t ev[7];
        for (int i = 0; i < 7; ++i) CU(cudaEventCreate(&ev[i]));
        for (int i = 0; i < CFD_PROFILE_KERNELS; ++i) ms[i] = 0.0;
        const int order[6] = {0, 1, 2, 3, 4, 5};
        cfd_status st = CFD_OK;
        for (int r = 0; r < reps && st == CFD_OK; ++r) {
            st = ctx->prm.precision == CFD_FP32_BULK ? enqueue_batch_stage<float>(ctx, 0, ev)
                                                     : enqueue_batch_stage<double>(ctx, 0, ev);
            if (st != CFD_OK) break;
            CU(cudaEventSynchronize(ev[6]));
            for (int i = 0; i < 6; ++i) {
                float t = 0.0f;
                CU(cudaEventElapsedTime(&t, ev[order[i]], ev[order[i] + 1]));
                ms[i] += t / reps;
            }
        }
        for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
        return st;
    }
    {
        cfd_status st0 = autotune(ctx);
        if (st0 != CFD_OK) return st0;
    }
    cudaEvent_t ev[7];
    for (int i = 0; i < 7; ++i) CU(cudaEventCreate(&ev[i]));
    for (int i = 0; i < CFD_PROFILE_KERNELS; ++i) ms[i] = 0.0;
    cfd_status st = CFD_OK;
    for (int r = 0; r < reps && st == CFD_OK; ++r) {
        st = run_stage<EP_FINAL_RHS>(ctx, ctx->b.U, nullptr, nullptr, ctx->b.Uk, 0.0, 1.0, ev);
        if (st != CFD_OK) break;
        CU(cudaEventSynchronize(ev[6]));
        for (int i = 0; i < 6; ++i) {
            float t = 0.0f;
            CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms[i] += t / reps;
        }
    }
    for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
    if (st != CFD_OK) return st;
    return read_err(ctx);
}

// ---------------------------------------------------------------------------
// Allocation-free right-hand side (cfd_rhs_noalloc).  Every intermediate
// array lives in one file-scope device array; host code must not use the
// array's name as a device address (in host code it names a host-side
// stand-in), so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
// ---------------------------------------------------------------------------
namespace noalloc {

constexpr long long kMaxNodes = CFD_NOALLOC_MAX_NODES;
constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kMetOff = 0;
constexpr size_t kPOff = kMetOff + up((size_t)M_COUNT * kMaxNodes * sizeof(double));
constexpr size_t kFvOff = kPOff + up((size_t)7 * kMaxNodes * sizeof(double));
constexpr size_t kROff = kFvOff + up((size_t)12 * kMaxNodes * sizeof(double));
constexpr size_t kClsOff = kROff + up((size_t)5 * kMaxNodes * sizeof(double));
constexpr size_t kErrOff = kClsOff + up((size_t)kMaxNodes);
constexpr size_t kBytes = kErrOff + kAlign;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kBytes];

static std::mutex g_mu;
static unsigned char* g_dev_ptr[kMaxDevices];   // device address of g_scratch per device

// once per device, with that device current
static cudaError_t setup(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        const int smem = (int)stream_smem_bytes<double>();
        e = cudaFuncSetAttribute(k_sweep_s<double, 1, EP_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_sweep_s<double, 2, EP_FINAL_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = (unsigned char*)p;
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

static void fill_phys(Phys& ph, const cfd_params& p)
{
    ph = Phys{};
    ph.gamma = p.gamma;
    ph.gm1 = p.gamma - 1.0;
    ph.inv_gm1 = 1.0 / (p.gamma - 1.0);
    ph.Ma = p.Ma;
    ph.gMa2 = p.gamma * p.Ma * p.Ma;
    ph.inv2g = 1.0 / (2.0 * p.gamma);
    ph.invMa = 1.0 / p.Ma;
    ph.viscous = p.Re > 0.0;
    ph.invRe = p.Re > 0.0 ? 1.0 / p.Re : 0.0;
    ph.kcoef = p.Re > 0.0 ? 1.0 / ((p.gamma - 1.0) * p.Ma * p.Ma * p.Pr * p.Re) : 0.0;
    ph.Tw = p.T_wall;
    ph.visc_law = p.visc_law;
    ph.omega = p.visc_omega;
    ph.suth_s = p.visc_law == CFD_SUTHERLAND ? 110.4 / p.T_ref : 0.0;
    ph.scheme = p.scheme;
    ph.charrec = p.recon_vars == CFD_RECON_CHARACTERISTIC;
    ph.th1 = p.theta1;
    ph.th2 = p.theta2;
    ph.eps = p.weno_eps;
    ph.vorder = p.visc_order;
}

}  // namespace noalloc

extern "C" cfd_status cfd_eval_viscosity(const cfd_params* params, const double* T, double* mu, int n)
{
    if (!params || !T || !mu || n < 0) return fail(nullptr, CFD_EINVAL, "bad argument to cfd_eval_viscosity");
    if (params->visc_law != CFD_SUTHERLAND && params->visc_law != CFD_POWER)
        return fail(nullptr, CFD_EINVAL, "bad visc_law");
    if (params->visc_law == CFD_SUTHERLAND && !(params->T_ref > 0.0))
        return fail(nullptr, CFD_EINVAL, "T_ref must be > 0");
    if (n == 0) return CFD_OK;
    Phys ph;
    noalloc::fill_phys(ph, *params);
    fill_float_consts(ph);
    std::vector<double> td;
    std::vector<float> tf;
    power_tables(ph.omega, td, tf, ph.pc, ph.pcf);
    const size_t bd = td.size() * sizeof(double), bf = tf.size() * sizeof(float), bn = (size_t)n * sizeof(double);
    char* buf = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&buf, bd + bf + 2 * bn);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf, td.data(), bd, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + bd, tf.data(), bf, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + bd + bf, T, bn, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        ph.powtab = (const double*)buf;
        ph.powtabf = (const float*)(buf + bd);
        const double* dT = (const double*)(buf + bd + bf);
        double* dmu = (double*)(buf + bd + bf + bn);
        const int blocks = (n + 255) / 256;
        if (params->precision == CFD_FP32_BULK) k_eval_viscosity<float><<<blocks, 256, 0, st>>>(ph, dT, dmu, n);
        else k_eval_viscosity<double><<<blocks, 256, 0, st>>>(ph, dT, dmu, n);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(mu, dmu, bn, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (buf) cudaFree(buf);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(nullptr, CFD_ECUDA, std::string("viscosity evaluation: ") + cudaGetErrorString(e));
    return CFD_OK;
}

extern "C" cfd_status cfd_rhs_noalloc(const cfd_grid* grid, const cfd_params* params, const double* metrics,
                                      const double* U, double* dUdt, void* stream)
{
    using namespace noalloc;
    if (!grid || !params || !metrics || !U || !dUdt)
        return fail(nullptr, CFD_EINVAL, "null argument to cfd_rhs_noalloc");
    cfd_status st = validate(nullptr, grid, params);
    if (st != CFD_OK) return st;
    if (params->precision != CFD_FP64)
        return fail(nullptr, CFD_EUNSUPPORTED, "cfd_rhs_noalloc computes in FP64 only");
    if (params->recon_vars != CFD_RECON_COMPONENT)
        return fail(nullptr, CFD_EUNSUPPORTED, "cfd_rhs_noalloc reconstructs component-wise only");
    if (params->sensor != CFD_SENSOR_PLAIN)
        return fail(nullptr, CFD_EUNSUPPORTED, "cfd_rhs_noalloc has no learned-sensor weights: plain sensor only");
    if (params->metric_mode != CFD_METRIC_NODAL)
        return fail(nullptr, CFD_EUNSUPPORTED, "cfd_rhs_noalloc evaluates the nodal metric mode only");
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > kMaxNodes)
        return fail(nullptr, CFD_ENOMEM, "cfd_rhs_noalloc: grid has more than CFD_NOALLOC_MAX_NODES nodes");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(nullptr, CFD_ECUDA, "cfd_rhs_noalloc: no usable CUDA device");
    unsigned char* base = nullptr;
    e = setup(dev, &base);
    if (e != cudaSuccess) return fail(nullptr, CFD_ECUDA, std::string("cfd_rhs_noalloc set-up: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;

    Geo g{};
    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.N = N;
    for (int d = 0; d < 3; ++d) {
        g.per[d] = grid->bc_lo[d] == CFD_BC_PERIODIC;
        g.bc_lo[d] = grid->bc_lo[d];
        g.bc_hi[d] = grid->bc_hi[d];
    }
    g.mlayout = grid->metric_layout;
    g.M = g.mlayout == CFD_METRICS_3D ? N : (g.mlayout == CFD_METRICS_2D ? (long long)g.nx * g.ny : 1);
    double* met = (double*)(base + kMetOff);
    g.met = met;
    Phys ph;
    fill_phys(ph, *params);
    void* P = base + kPOff;
    void* Fv = base + kFvOff;
    void* R = base + kROff;
    uint8_t* cls = base + kClsOff;
    int* err = (int*)(base + kErrOff);

#define NA_CHECK(x)                                                                                       \
    do {                                                                                                  \
        cudaError_t e_ = (x);                                                                             \
        if (e_ != cudaSuccess) return fail(nullptr, CFD_ECUDA, std::string("cfd_rhs_noalloc: ") + cudaGetErrorString(e_)); \
    } while (0)
    // the caller's metrics into the array, then the derived quantities
    NA_CHECK(cudaMemcpyAsync(met, metrics, 10 * g.M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_metric_derive<<<grid_for(g.M, 256), 256, 0, s>>>(met, g.M);
    NA_CHECK(cudaGetLastError());
    // the only value that must start at zero; every other array is fully
    // written before it is read
    NA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), s));
    SweepArgs A{};
    A.g = g;
    A.ph = ph;
    A.P = P;
    A.cls = params->scheme == CFD_HYBRID ? cls : nullptr;
    A.cls_io = cls;
    A.Fv = ph.viscous ? Fv : nullptr;
    A.R = R;
    A.err = err;
    A.U = U;
    A.Lout = dUdt;
    A.rk_b = 1.0;
    A.seg_len = 128;
    const NodeLaunch nl = node_launch(g);
    k_prim<double><<<nl.grid, nl.block, 0, s>>>(A);
    NA_CHECK(cudaGetLastError());
    if (params->scheme == CFD_HYBRID) {
        k_sensor<<<nl.grid, nl.block, 0, s>>>(A);
        NA_CHECK(cudaGetLastError());
    }
    if (ph.viscous) {
        k_visc_flux<double><<<nl.grid, nl.block, 0, s>>>(A);
        NA_CHECK(cudaGetLastError());
    }
    {
        const int lo = g.per[0] ? 0 : 1, hi = g.per[0] ? g.nx : g.nx - 1;
        const int nb = g.nx <= 32 ? 32 : (g.nx <= 64 ? 64 : 128);
        dim3 gr((hi - lo + nb - 1) / nb, g.ny, g.nz);
        if (nb == 32) k_sweep_x<double, 32, EP_STORE><<<gr, 32, 0, s>>>(A);
        else if (nb == 64) k_sweep_x<double, 64, EP_STORE><<<gr, 64, 0, s>>>(A);
        else k_sweep_x<double, 128, EP_STORE><<<gr, 128, 0, s>>>(A);
        NA_CHECK(cudaGetLastError());
    }
    const size_t smem = stream_smem_bytes<double>();
    {
        const int lo = g.per[1] ? 0 : 1, hi = g.per[1] ? g.ny : g.ny - 1;
        const long long nseg = (hi - lo + A.seg_len - 1) / A.seg_len;
        const long long warps = (long long)((g.nx + 31) / 32) * g.nz * nseg;
        k_sweep_s<double, 1, EP_ACCUM><<<(unsigned)((warps + 3) / 4), 128, smem, s>>>(A);
        NA_CHECK(cudaGetLastError());
    }
    {
        const int lo = g.per[2] ? 0 : 1, hi = g.per[2] ? g.nz : g.nz - 1;
        const long long nseg = (hi - lo + A.seg_len - 1) / A.seg_len;
        const long long warps = (long long)((g.nx + 31) / 32) * g.ny * nseg;
        k_sweep_s<double, 2, EP_FINAL_RHS><<<(unsigned)((warps + 3) / 4), 128, smem, s>>>(A);
        NA_CHECK(cudaGetLastError());
    }
#undef NA_CHECK
    return CFD_OK;
}

// ---------------------------------------------------------------------------
// learned sensor: weights, features, fallback statistics
// ---------------------------------------------------------------------------
extern "C" cfd_status cfd_set_sensor_mlp(cfd_ctx* ctx, const void* weights_bf16, const float* biases, float conf_min)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    // an ensemble: every block gets the weights (its per-block calls run on
    // the block's own context), the ensemble's step uses its own copy
    for (cfd_ctx* sb : ctx->sub) {
        const cfd_status st = cfd_set_sensor_mlp(sb, weights_bf16, biases, conf_min);
        if (st != CFD_OK) {
            ctx->msg = sb->msg;
            return st;
        }
    }
    if (!weights_bf16 || !biases) {
        ctx->mlp_on = false;
        ctx->prm.sensor = CFD_SENSOR_PLAIN;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    if (!(conf_min >= 0.0f && conf_min <= 1.0f)) return fail(ctx, CFD_EINVAL, "conf_min must be in [0, 1]");
    // padded layouts: w1 [32][48], w2 [32][32], w3 [8][32]; biases b1[32], b2[32], b3[8]
    const size_t n1 = 32 * MLP_KP, n2 = 32 * 32, n3 = 8 * 32;
    std::vector<uint16_t> hw(n1 + n2 + n3, 0);
    const uint16_t* src = (const uint16_t*)weights_bf16;
    for (int o = 0; o < 32; ++o)
        for (int i = 0; i < MLP_IN; ++i) hw[o * MLP_KP + i] = src[o * MLP_IN + i];
    src += 32 * MLP_IN;
    for (int o = 0; o < 32; ++o)
        for (int i = 0; i < 32; ++i) hw[n1 + o * 32 + i] = src[o * 32 + i];
    src += 32 * 32;
    for (int o = 0; o < MLP_OUT; ++o)
        for (int i = 0; i < 32; ++i) hw[n1 + n2 + o * 32 + i] = src[o * 32 + i];
    std::vector<float> hb(72, 0.0f);
    for (int e = 0; e < 32; ++e) hb[e] = biases[e];
    for (int e = 0; e < 32; ++e) hb[32 + e] = biases[32 + e];
    for (int e = 0; e < MLP_OUT; ++e) hb[64 + e] = biases[64 + e];
    const size_t wbytes = hw.size() * sizeof(uint16_t), bbytes = hb.size() * sizeof(float);
    if (!ctx->mlp_buf) CU(cudaMalloc(&ctx->mlp_buf, wbytes + bbytes + 64));
    char* base = (char*)ctx->mlp_buf;
    CU(cudaMemcpyAsync(base, hw.data(), wbytes, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(base + wbytes, hb.data(), bbytes, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(base + wbytes + bbytes, 0, 8, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const uint16_t* dw = (const uint16_t*)base;
    const float* db = (const float*)(base + wbytes);
    ctx->mlp = MlpArgs{dw, dw + n1, dw + n1 + n2, db, db + 32, db + 64, conf_min,
                       (unsigned long long*)(base + wbytes + bbytes)};
    ctx->mlp_on = true;
    ctx->prm.sensor = CFD_SENSOR_MLP;
    ctx->graph_valid = false;
    return CFD_OK;
}

extern "C" cfd_status cfd_sensor_features(cfd_ctx* ctx, int block, float* out, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    if (!out) return fail(ctx, CFD_EINVAL, "null output");
    DELEGATE(cfd_sensor_features(b_, 0, out, on_device));
    const Geo& g = ctx->g;
    const long long bytes = (long long)MLP_IN * g.N * sizeof(float);
    float* dev = nullptr;
    if (on_device) {
        dev = out;
    } else {
        CU(cudaMalloc(&dev, bytes));
    }
    const NodeLaunch nl = node_launch(g);
    const SweepArgs A = make_args(ctx, ctx->b.U, nullptr, nullptr, nullptr, 0.0, 1.0);
    if (ctx->prm.precision == CFD_FP32_BULK)
        k_prim_mixed<<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    else
        k_prim<double><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    LAUNCH_CHECK();
    if (ctx->prm.precision == CFD_FP32_BULK)
        k_mlp_features<float><<<nl.grid, nl.block, 0, ctx->stream>>>(A, dev);
    else
        k_mlp_features<double><<<nl.grid, nl.block, 0, ctx->stream>>>(A, dev);
    LAUNCH_CHECK();
    if (!on_device) {
        CU(cudaMemcpyAsync(out, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        cudaFree(dev);
    }
    return read_err(ctx);
}

extern "C" cfd_status cfd_sensor_fallbacks(cfd_ctx* ctx, unsigned long long* count)
{
    if (!ctx || !count) return fail(ctx, CFD_EINVAL, "null argument");
    *count = 0;
    if (!ctx->mlp_on) return CFD_OK;
    CU(cudaMemcpyAsync(ctx->h_pinned + 5, ctx->mlp.fallbacks, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp.fallbacks, 0, 8, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    std::memcpy(count, ctx->h_pinned + 5, 8);
    return CFD_OK;
}
