// cfd_api.cu -- the C ABI (include/cfd.h): context, device buffers, stage
// orchestration and CUDA-graph replay of the TVD-RK3 step (Eq. 45).
#include <cuda_runtime.h>

#include <chrono>
#include <mutex>
#include <vector>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>

#include "../../include/cfd.h"
#include "cfd_kernels.cuh"

using namespace cfdk;

namespace {

constexpr int kSMs = 152;

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
    MlpArgs mlp{};
    bool mlp_on = false;              // 0 node-parallel, 1 2.5-D TZ 64, 2 2.5-D TZ 32 (autotuned)
    bool tuned = false;
    // ensemble of blocks (cfd_create_batch): one single-block context per block
    // plus the tables that drive one persistent launch per kernel kind
    std::vector<cfd_ctx*> sub;
    SweepArgs* d_tbl[3] = {nullptr, nullptr, nullptr};  // per stage, [nb]
    int* d_maps = nullptr;                              // all prefix / gdim arrays
    BatchMap maps[3][5];                                // [stage][kind]
    int map_grid[5] = {0, 0, 0, 0, 0};                  // persistent grid per kind
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
            if (t < 0 || t > 4) return fail(ctx, CFD_EINVAL, "unknown boundary condition");
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
    if (p->metric_mode != CFD_METRIC_NODAL) return fail(ctx, CFD_EUNSUPPORTED, "only the nodal metric mode");
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
                    c->mlp_buf,
                    c->cflmax, c->inflow, c->wall_x, c->wall_z};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
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
static cfd_status launch_bc(cfd_ctx* ctx, double* U, double tfrac, bool use_dt)
{
    const Geo& g = ctx->g;
    for (int d = 0; d < 3; ++d) {
        if (g.per[d]) continue;
        long long nface = d == 0 ? (long long)g.ny * g.nz : (d == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny);
        k_bc<<<grid_for(2 * nface, 256), 256, 0, ctx->stream>>>(g, ctx->ph, ctx->bc, U, d, ctx->t,
                                                                  use_dt ? ctx->dt : nullptr, tfrac);
        LAUNCH_CHECK();
    }
    return CFD_OK;
}

template <class R>
static cfd_status launch_visc(cfd_ctx* ctx, const SweepArgs& A, int kind)
{
    const Geo& g = ctx->g;
    if (kind == 0) {
        const NodeLaunch nl = node_launch(g);
        k_visc_flux<R><<<nl.grid, nl.block, 0, ctx->stream>>>(A);
    } else if (kind == 3) {
        dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
        k_visc_flux<R, 4><<<grid, dim3(32, 4), 0, ctx->stream>>>(A);
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
    } else if (kind == 2) {
        const int seg = param > 0 ? param : std::max(1, hi - lo);
        A.seg_len = seg;
        dim3 grid((g.nx + 31) / 32, nother, (hi - lo + seg - 1) / seg);
        k_sweep_w<R, DIR, EP><<<grid, 256, walk_smem_bytes<R>(), ctx->stream>>>(A);
    } else {
        dim3 grid((g.nx + 31) / 32, nother, (hi - lo + param - 1) / param);
        if (param == 16)
            k_sweep_t<R, DIR, EP, 16><<<grid, 256, tile_smem_bytes<R, 16>(), ctx->stream>>>(A);
        else
            k_sweep_t<R, DIR, EP, 32><<<grid, 256, tile_smem_bytes<R, 32>(), ctx->stream>>>(A);
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
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_w<R, DIR, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)walk_smem_bytes<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_w<R, DIR, EP>, cudaFuncAttributePreferredSharedMemoryCarveout,
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
    if (!ctx->forced && (mixed || ctx->prm.scheme == CFD_HYBRID)) {
        if (ctx->prm.sensor == CFD_SENSOR_MLP) {
            if (!ctx->mlp_on) return fail(ctx, CFD_EINVAL, "learned sensor selected but no weights set");
            dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
            k_sensor_mlp<R><<<grid, 128, 0, ctx->stream>>>(A, ctx->mlp);
        } else if (mixed) {
            k_sensor32<<<nl.grid, nl.block, 0, ctx->stream>>>(A);
        } else {
            k_sensor<<<nl.grid, nl.block, 0, ctx->stream>>>(A);
        }
        LAUNCH_CHECK();
    }
    if (ev) cudaEventRecord(ev[2], ctx->stream);
    if (ctx->ph.viscous) {
        cfd_status st = launch_visc<R>(ctx, A, ctx->visc_kind);
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
namespace {
struct TuneKey {
    int prec, nx, ny, nz, per0, per1, per2, scheme, viscous;
    bool operator==(const TuneKey& o) const
    {
        return prec == o.prec && nx == o.nx && ny == o.ny && nz == o.nz && per0 == o.per0 && per1 == o.per1 &&
               per2 == o.per2 && scheme == o.scheme && viscous == o.viscous;
    }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, std::vector<int>>> g_tune_cache;
}  // namespace

static TuneKey tune_key(const cfd_ctx* ctx)
{
    return {ctx->prm.precision, ctx->g.nx, ctx->g.ny, ctx->g.nz, ctx->g.per[0], ctx->g.per[1], ctx->g.per[2],
            ctx->prm.scheme, ctx->ph.viscous};
}

template <class R>
static cfd_status autotune_t(cfd_ctx* ctx)
{
    cfd_status st = run_stage<EP_FINAL_RHS>(ctx, ctx->b.U, nullptr, nullptr, ctx->b.Uk, 0.0, 1.0);
    if (st != CFD_OK) return st;
    SweepArgs A = make_args(ctx, ctx->b.U, nullptr, nullptr, ctx->b.Uk, 0.0, 1.0);
    const int cands[6][2] = {{0, 128}, {0, 64}, {1, 32}, {1, 16}, {2, 0}, {2, 64}};
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int dir = 1; dir <= 2 && st == CFD_OK; ++dir) {
        float best = 1e30f;
        for (int c = 0; c < 6 && st == CFD_OK; ++c) {
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
        float best = 1e30f;
        for (int kind = 0; kind < 4 && st == CFD_OK; ++kind) {
            for (int rep = 0; rep < 4 && st == CFD_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, ctx->stream);
                st = launch_visc<R>(ctx, A, kind);
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
    const TuneKey key = tune_key(ctx);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto& kv : g_tune_cache)
            if (kv.first == key) {
                for (int d = 1; d <= 2; ++d) {
                    ctx->sweep_kind[d] = kv.second[2 * d - 2];
                    ctx->sweep_param[d] = kv.second[2 * d - 1];
                }
                ctx->visc_kind = kv.second[4];
                ctx->xi_kind = kv.second[5];
                ctx->xi_seg = kv.second[6];
                ctx->tuned = true;
                return CFD_OK;
            }
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
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back(
        {key, {ctx->sweep_kind[1], ctx->sweep_param[1], ctx->sweep_kind[2], ctx->sweep_param[2], ctx->visc_kind,
               ctx->xi_kind, ctx->xi_seg}});
    return CFD_OK;
}

extern "C" cfd_status cfd_set_sweep_variant(cfd_ctx* ctx, int dir, int kind, int param)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
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
    if (dir < 1 || dir > 2 || kind < 0 || kind > 2) return fail(ctx, CFD_EINVAL, "dir must be 0, 1, 2 or 3");
    if (kind == 1 && param != 16 && param != 32) return fail(ctx, CFD_EINVAL, "tile length must be 16 or 32");
    if (kind == 0 && (param < 1 || param > 65535)) return fail(ctx, CFD_EINVAL, "segment length out of range");
    if (kind == 2 && (param < 0 || param > 65535)) return fail(ctx, CFD_EINVAL, "segment length out of range");
    ctx->sweep_kind[dir] = kind;
    ctx->sweep_param[dir] = param;
    ctx->tuned = true;
    ctx->graph_valid = false;
    return CFD_OK;
}

extern "C" cfd_status cfd_get_sweep_variant(cfd_ctx* ctx, int dir, int* kind, int* param)
{
    if (!ctx || !kind || !param || dir < 0 || dir > 3) return fail(ctx, CFD_EINVAL, "bad argument");
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
enum { MK_NODE = 0, MK_VISC = 1, MK_SX = 2, MK_T1 = 3, MK_T2 = 4, MK_COUNT = 5 };
constexpr int kBatchBX = 64, kBatchTL = 16, kBatchTZ = 32;

static void batch_tiles(const Geo& g, int kind, int out[3])
{
    auto cdiv = [](int a, int b) { return (a + b - 1) / b; };
    auto span = [&](int d) {
        const int n = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
        return g.per[d] ? n : n - 2;
    };
    switch (kind) {
    case MK_NODE: out[0] = (int)((g.N + 127) / 128); out[1] = 1; out[2] = 1; break;  // flat node runs
    case MK_VISC: out[0] = cdiv(g.nx, 32); out[1] = cdiv(g.ny, 8); out[2] = cdiv(g.nz, kBatchTZ); break;
    case MK_SX: out[0] = cdiv(span(0), kBatchBX); out[1] = g.ny; out[2] = g.nz; break;
    case MK_T1: out[0] = cdiv(g.nx, 32); out[1] = g.nz; out[2] = cdiv(span(1), kBatchTL); break;
    default: out[0] = cdiv(g.nx, 32); out[1] = g.ny; out[2] = cdiv(span(2), kBatchTL); break;
    }
}

template <class R>
static cudaError_t batch_kernel_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(kb_visc_flux25<R, kBatchTZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)visc25_smem_bytes<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 1, EP_ACCUM, kBatchTL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, kBatchTL>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 2, EP_FINAL_RK, kBatchTL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, kBatchTL>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 1, EP_ACCUM, kBatchTL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_sweep_t<R, 2, EP_FINAL_RK, kBatchTL>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
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

template <class R>
static void batch_grids(cfd_ctx* ctx, const int totals[MK_COUNT])
{
    const bool mixed = sizeof(R) == sizeof(float);
    ctx->map_grid[MK_NODE] = mixed ? persistent_grid(kb_prim_mixed, 128, 0, totals[MK_NODE])
                                   : persistent_grid(kb_prim<double>, 128, 0, totals[MK_NODE]);
    ctx->map_grid[MK_VISC] = persistent_grid(kb_visc_flux25<R, kBatchTZ>, 256, visc25_smem_bytes<R>(), totals[MK_VISC]);
    ctx->map_grid[MK_SX] = persistent_grid(kb_sweep_x<R, kBatchBX, EP_STORE>, kBatchBX, 0, totals[MK_SX]);
    ctx->map_grid[MK_T1] = persistent_grid(kb_sweep_t<R, 1, EP_ACCUM, kBatchTL>, 256, tile_smem_bytes<R, kBatchTL>(),
                                           totals[MK_T1]);
    ctx->map_grid[MK_T2] = persistent_grid(kb_sweep_t<R, 2, EP_FINAL_RK, kBatchTL>, 256,
                                           tile_smem_bytes<R, kBatchTL>(), totals[MK_T2]);
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
        }
        CU(cudaMalloc(&ctx->d_tbl[s], nb * sizeof(SweepArgs)));
        CU(cudaMemcpyAsync(ctx->d_tbl[s], tbl.data(), nb * sizeof(SweepArgs), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    // work-list maps: prefix sums of tiles and per-block tile grids per kernel kind
    const int per_kind = (nb + 1) + 3 * nb;
    std::vector<int> h((size_t)MK_COUNT * per_kind);
    int totals[MK_COUNT];
    for (int k = 0; k < MK_COUNT; ++k) {
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
        for (int k = 0; k < MK_COUNT; ++k) {
            int* pre = ctx->d_maps + (size_t)k * per_kind;
            ctx->maps[s][k] = BatchMap{ctx->d_tbl[s], pre, pre + nb + 1, nb};
        }
    if (params[0].precision == CFD_FP32_BULK) {
        CU((batch_kernel_attrs<float>()));
        batch_grids<float>(ctx, totals);
    } else {
        CU((batch_kernel_attrs<double>()));
        batch_grids<double>(ctx, totals);
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

template <class R>
static cfd_status enqueue_batch_stage(cfd_ctx* ctx, int s, cudaEvent_t* ev)
{
    const bool mixed = sizeof(R) == sizeof(float);
    const cudaStream_t st = ctx->stream;
    const BatchMap* m = ctx->maps[s];
    if (ev) cudaEventRecord(ev[0], st);
    if (mixed) kb_prim_mixed<<<ctx->map_grid[MK_NODE], 128, 0, st>>>(m[MK_NODE]);
    else kb_prim<double><<<ctx->map_grid[MK_NODE], 128, 0, st>>>(m[MK_NODE]);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[1], st);
    if (mixed || ctx->prm.scheme == CFD_HYBRID) {
        if (mixed) kb_sensor32<<<ctx->map_grid[MK_NODE], 128, 0, st>>>(m[MK_NODE]);
        else kb_sensor<<<ctx->map_grid[MK_NODE], 128, 0, st>>>(m[MK_NODE]);
        LAUNCH_CHECK();
    }
    if (ev) cudaEventRecord(ev[2], st);
    if (ctx->ph.viscous) {
        kb_visc_flux25<R, kBatchTZ><<<ctx->map_grid[MK_VISC], 256, visc25_smem_bytes<R>(), st>>>(m[MK_VISC]);
        LAUNCH_CHECK();
    }
    if (ev) cudaEventRecord(ev[3], st);
    kb_sweep_x<R, kBatchBX, EP_STORE><<<ctx->map_grid[MK_SX], kBatchBX, 0, st>>>(m[MK_SX]);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[4], st);
    kb_sweep_t<R, 1, EP_ACCUM, kBatchTL><<<ctx->map_grid[MK_T1], 256, tile_smem_bytes<R, kBatchTL>(), st>>>(m[MK_T1]);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[5], st);
    kb_sweep_t<R, 2, EP_FINAL_RK, kBatchTL><<<ctx->map_grid[MK_T2], 256, tile_smem_bytes<R, kBatchTL>(), st>>>(
        m[MK_T2]);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[6], st);
    // boundary conditions of blocks with non-periodic faces, at the stage time
    const double tfrac[3] = {1.0, 0.5, 1.0};
    for (cfd_ctx* sb : ctx->sub) {
        double* Uout = s == 2 ? sb->b.U : sb->b.Uk;
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
    st = launch_bc(ctx, ctx->b.Uk, 1.0, true);
    if (st != CFD_OK) return st;
    // stage 2: Uk = 3/4 U + 1/4 (Uk + dt L(Uk))
    st = run_stage<EP_FINAL_RK>(ctx, ctx->b.Uk, ctx->b.U, ctx->b.Uk, nullptr, 0.75, 0.25);
    if (st != CFD_OK) return st;
    st = launch_bc(ctx, ctx->b.Uk, 0.5, true);
    if (st != CFD_OK) return st;
    // stage 3: U = 1/3 U + 2/3 (Uk + dt L(Uk))
    st = run_stage<EP_FINAL_RK>(ctx, ctx->b.Uk, ctx->b.U, ctx->b.U, nullptr, 1.0 / 3.0, 2.0 / 3.0);
    if (st != CFD_OK) return st;
    st = launch_bc(ctx, ctx->b.U, 1.0, true);
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
            for (int d = 0; d < 3; ++d) per_stage += sb->g.per[d] ? 0 : 1;
        return 3 * per_stage + 1;
    }
    const bool sensor = !ctx->forced && (ctx->prm.scheme == CFD_HYBRID || ctx->prm.precision == CFD_FP32_BULK);
    long long per_stage = 1 + 3 + (sensor ? 1 : 0) + (ctx->ph.viscous ? 1 : 0);
    long long bc = 0;
    for (int d = 0; d < 3; ++d) bc += ctx->g.per[d] ? 0 : 1;
    return 3 * (per_stage + bc) + 1;
}

extern "C" cfd_status cfd_step(cfd_ctx* ctx, double dt, int nsteps)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    if (!(dt > 0.0) || nsteps < 0) return fail(ctx, CFD_EINVAL, "dt must be > 0 and nsteps >= 0");
    if (nsteps == 0) return CFD_OK;
    k_set_scalar<<<1, 32, 0, ctx->stream>>>(ctx->dt, dt);
    LAUNCH_CHECK();
    if (ctx->sub.empty()) {
        cfd_status st = autotune(ctx);
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
    if (!ctx->sub.empty()) return fail(ctx, CFD_EUNSUPPORTED, "the learned sensor is per single-block context");
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
