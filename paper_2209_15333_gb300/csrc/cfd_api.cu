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
    int sweep_kind[3] = {0, 0, 0};  // eta/zeta: 0 streaming, 1 tile (chosen by the autotuner)
    int sweep_param[3] = {0, 128, 128};
    int visc_kind = 0;              // 0 node-parallel, 1 2.5-D TZ 64, 2 2.5-D TZ 32 (autotuned)
    bool tuned = false;
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
            if (t < 0 || t > 3) return fail(ctx, CFD_EINVAL, "unknown boundary condition");
        }
        bool plo = gr->bc_lo[d] == CFD_BC_PERIODIC, phi = gr->bc_hi[d] == CFD_BC_PERIODIC;
        if (plo != phi) return fail(ctx, CFD_EINVAL, "periodic must be set on both faces of a direction");
        if (!plo && n[d] < 8) return fail(ctx, CFD_EINVAL, "non-periodic directions need >= 8 nodes");
        if (gr->bc_lo[d] == CFD_BC_INFLOW && d != 0) return fail(ctx, CFD_EINVAL, "inflow only on the xi-low face");
        if (gr->bc_hi[d] == CFD_BC_INFLOW) return fail(ctx, CFD_EINVAL, "inflow only on the xi-low face");
    }
    if (gr->ny > 65535 || gr->nz > 65535) return fail(ctx, CFD_EINVAL, "ny, nz must be <= 65535");
    if (gr->metric_layout < 0 || gr->metric_layout > 2) return fail(ctx, CFD_EINVAL, "bad metric_layout");
    if (!(p->gamma > 1.0) || !(p->Ma > 0.0)) return fail(ctx, CFD_EINVAL, "gamma must be > 1 and Ma > 0");
    if (p->Re > 0.0 && !(p->Pr > 0.0)) return fail(ctx, CFD_EINVAL, "Pr must be > 0");
    if (p->scheme < 0 || p->scheme > 3) return fail(ctx, CFD_EINVAL, "unknown scheme");
    if (p->visc_order != 6 && p->visc_order != 8) return fail(ctx, CFD_EINVAL, "visc_order must be 6 or 8");
    if (p->visc_law != CFD_SUTHERLAND && p->visc_law != CFD_POWER) return fail(ctx, CFD_EINVAL, "bad visc_law");
    if (p->visc_law == CFD_SUTHERLAND && !(p->T_ref > 0.0)) return fail(ctx, CFD_EINVAL, "T_ref must be > 0");
    if (!(p->weno_eps > 0.0)) return fail(ctx, CFD_EINVAL, "weno_eps must be > 0");
    if (p->metric_mode != CFD_METRIC_NODAL) return fail(ctx, CFD_EUNSUPPORTED, "only the nodal metric mode");
    if (p->precision != CFD_FP64 && p->precision != CFD_FP32_BULK) return fail(ctx, CFD_EINVAL, "unknown precision");
    if (p->sensor != CFD_SENSOR_PLAIN) return fail(ctx, CFD_EUNSUPPORTED, "only the plain sensor");
    if (p->scheme == CFD_HYBRID && !(p->theta1 <= p->theta2)) return fail(ctx, CFD_EINVAL, "theta1 > theta2");
    bool wall = false;
    for (int d = 0; d < 3; ++d) wall |= gr->bc_lo[d] == CFD_BC_WALL_ISOTHERMAL || gr->bc_hi[d] == CFD_BC_WALL_ISOTHERMAL;
    if (wall && !(p->T_wall > 0.0)) return fail(ctx, CFD_EINVAL, "T_wall must be > 0");
    return CFD_OK;
}

static void free_all(cfd_ctx* c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    void* ptrs[] = {c->b.U, c->b.Uk, c->b.P, c->b.Fv, c->b.R, c->b.cls, c->met, c->metf, c->err, c->dt, c->t,
                    c->cflmax, c->inflow, c->wall_x, c->wall_z};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
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
    Phys& ph = ctx->ph;
    const cfd_params& p = *params;
    ph.gamma = p.gamma;
    ph.gm1 = p.gamma - 1.0;
    ph.inv_gm1 = 1.0 / (p.gamma - 1.0);
    ph.Ma = p.Ma;
    ph.gMa2 = p.gamma * p.Ma * p.Ma;
    ph.inv2g = 1.0 / (2.0 * p.gamma);
    ph.viscous = p.Re > 0.0;
    ph.invRe = p.Re > 0.0 ? 1.0 / p.Re : 0.0;
    ph.kcoef = p.Re > 0.0 ? 1.0 / ((p.gamma - 1.0) * p.Ma * p.Ma * p.Pr * p.Re) : 0.0;
    ph.Tw = p.T_wall;
    ph.visc_law = p.visc_law;
    ph.omega = p.visc_omega;
    ph.suth_s = p.visc_law == CFD_SUTHERLAND ? 110.4 / p.T_ref : 0.0;
    ph.scheme = p.scheme;
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
    if (block != 0) return fail(ctx, CFD_EINVAL, "block index out of range");
    return CFD_OK;
}

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
static cfd_status launch_visc(cfd_ctx* ctx, int kind)
{
    const Geo& g = ctx->g;
    if (kind == 0) {
        const NodeLaunch nl = node_launch(g);
        k_visc_flux<R><<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, (const R*)ctx->b.P, (R*)ctx->b.Fv);
    } else {
        const int tz = kind == 1 ? 64 : 32;
        dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + tz - 1) / tz);
        if (kind == 1)
            k_visc_flux25<R, 64><<<grid, 256, visc25_smem_bytes<R>(), ctx->stream>>>(g, ctx->ph, (const R*)ctx->b.P,
                                                                                   (R*)ctx->b.Fv);
        else
            k_visc_flux25<R, 32><<<grid, 256, visc25_smem_bytes<R>(), ctx->stream>>>(g, ctx->ph, (const R*)ctx->b.P,
                                                                                   (R*)ctx->b.Fv);
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
    if (kind == 0) {
        A.seg_len = param;
        const long long nseg = (hi - lo + param - 1) / param;
        const long long warps = (long long)((g.nx + 31) / 32) * nother * nseg;
        k_sweep_s<R, DIR, EP><<<(unsigned)((warps + 3) / 4), 128, 4 * 80 * 32 * sizeof(R), ctx->stream>>>(A);
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

template <class R, int EPF>
static cfd_status launch_sweeps(cfd_ctx* ctx, SweepArgs& A, cudaEvent_t* ev = nullptr)
{
    const Geo& g = ctx->g;
    // xi
    {
        int lo = g.per[0] ? 0 : 1, hi = g.per[0] ? g.nx : g.nx - 1;
        int nb = ctx->bx;
        dim3 grid((hi - lo + nb - 1) / nb, g.ny, g.nz);
        if (nb == 32) k_sweep_x<R, 32, EP_STORE><<<grid, 32, 0, ctx->stream>>>(A);
        else if (nb == 64) k_sweep_x<R, 64, EP_STORE><<<grid, 64, 0, ctx->stream>>>(A);
        else k_sweep_x<R, 128, EP_STORE><<<grid, 128, 0, ctx->stream>>>(A);
        LAUNCH_CHECK();
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
                                         (int)(4 * 80 * 32 * sizeof(R)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, 16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_t<R, DIR, EP, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<R, 32>());
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
    A.Fv = ctx->ph.viscous ? ctx->b.Fv : nullptr;
    A.R = ctx->b.R;
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
    const long long N = g.N;
    const bool mixed = sizeof(R) == sizeof(float);
    if (ev) cudaEventRecord(ev[0], ctx->stream);
    const NodeLaunch nl = node_launch(g);
    if (mixed)
        k_prim_mixed<<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, Uin, (float*)ctx->b.P, ctx->b.cls, ctx->err);
    else
        k_prim<double><<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, Uin, (double*)ctx->b.P, ctx->err);
    LAUNCH_CHECK();
    if (ev) cudaEventRecord(ev[1], ctx->stream);
    if (!ctx->forced && (mixed || ctx->prm.scheme == CFD_HYBRID)) {
        if (mixed)
            k_sensor32<<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, (const float*)ctx->b.P + 4 * N, ctx->b.cls);
        else
            k_sensor<<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, (const double*)ctx->b.P + 4 * N, ctx->b.cls);
        LAUNCH_CHECK();
    }
    if (ev) cudaEventRecord(ev[2], ctx->stream);
    if (ctx->ph.viscous) {
        cfd_status st = launch_visc<R>(ctx, ctx->visc_kind);
        if (st != CFD_OK) return st;
    }
    SweepArgs A = make_args(ctx, Uin, Un, Uout, Lout, a, b);
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
    const int cands[4][2] = {{0, 128}, {0, 64}, {1, 32}, {1, 16}};
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int dir = 1; dir <= 2 && st == CFD_OK; ++dir) {
        float best = 1e30f;
        for (int c = 0; c < 4 && st == CFD_OK; ++c) {
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
    if (ctx->ph.viscous) {
        float best = 1e30f;
        for (int kind = 0; kind < 3 && st == CFD_OK; ++kind) {
            for (int rep = 0; rep < 4 && st == CFD_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, ctx->stream);
                st = launch_visc<R>(ctx, kind);
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
                ctx->tuned = true;
                return CFD_OK;
            }
    }
    cfd_status st = ctx->prm.precision == CFD_FP32_BULK ? autotune_t<float>(ctx) : autotune_t<double>(ctx);
    if (st != CFD_OK) return st;
    ctx->tuned = true;
    ctx->graph_valid = false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back(
        {key, {ctx->sweep_kind[1], ctx->sweep_param[1], ctx->sweep_kind[2], ctx->sweep_param[2], ctx->visc_kind}});
    return CFD_OK;
}

extern "C" cfd_status cfd_set_sweep_variant(cfd_ctx* ctx, int dir, int kind, int param)
{
    if (!ctx) return fail(nullptr, CFD_EINVAL, "null context");
    if (dir == 0) {
        if (kind < 0 || kind > 2) return fail(ctx, CFD_EINVAL, "viscous kernel kind must be 0, 1 or 2");
        ctx->visc_kind = kind;
        ctx->tuned = true;
        ctx->graph_valid = false;
        return CFD_OK;
    }
    if (dir < 1 || dir > 2 || kind < 0 || kind > 1) return fail(ctx, CFD_EINVAL, "dir must be 0, 1 or 2");
    if (kind == 1 && param != 16 && param != 32) return fail(ctx, CFD_EINVAL, "tile length must be 16 or 32");
    if (kind == 0 && (param < 1 || param > 65535)) return fail(ctx, CFD_EINVAL, "segment length out of range");
    ctx->sweep_kind[dir] = kind;
    ctx->sweep_param[dir] = param;
    ctx->tuned = true;
    ctx->graph_valid = false;
    return CFD_OK;
}

extern "C" cfd_status cfd_get_sweep_variant(cfd_ctx* ctx, int dir, int* kind, int* param)
{
    if (!ctx || !kind || !param || dir < 0 || dir > 2) return fail(ctx, CFD_EINVAL, "bad argument");
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

extern "C" cfd_status cfd_set_state(cfd_ctx* ctx, int block, const double* U, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
    if (!U) return fail(ctx, CFD_EINVAL, "null state");
    const long long N = ctx->g.N;
    CU(cudaMemcpyAsync(ctx->b.U, U, 5 * N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
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
    if (!U) return fail(ctx, CFD_EINVAL, "null output");
    const long long N = ctx->g.N;
    CU(cudaMemcpyAsync(U, ctx->b.U, 5 * N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    return read_err(ctx);
}

extern "C" cfd_status cfd_rhs(cfd_ctx* ctx, int block, double* dUdt, int on_device)
{
    cfd_status st = check_block(ctx, block);
    if (st != CFD_OK) return st;
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

static cfd_status enqueue_step(cfd_ctx* ctx)
{
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
    {
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
    if (!dt || !(cfl > 0.0)) return fail(ctx, CFD_EINVAL, "bad cfl or null output");
    const Geo& g = ctx->g;
    const bool mixed = ctx->prm.precision == CFD_FP32_BULK;
    const NodeLaunch nl = node_launch(g);
    if (mixed)
        k_prim_mixed<<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, ctx->b.U, (float*)ctx->b.P, ctx->b.cls, ctx->err);
    else
        k_prim<double><<<nl.grid, nl.block, 0, ctx->stream>>>(g, ctx->ph, ctx->b.U, (double*)ctx->b.P, ctx->err);
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
        const int smem = 4 * 80 * 32 * (int)sizeof(double);
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
    ph.viscous = p.Re > 0.0;
    ph.invRe = p.Re > 0.0 ? 1.0 / p.Re : 0.0;
    ph.kcoef = p.Re > 0.0 ? 1.0 / ((p.gamma - 1.0) * p.Ma * p.Ma * p.Pr * p.Re) : 0.0;
    ph.Tw = p.T_wall;
    ph.visc_law = p.visc_law;
    ph.omega = p.visc_omega;
    ph.suth_s = p.visc_law == CFD_SUTHERLAND ? 110.4 / p.T_ref : 0.0;
    ph.scheme = p.scheme;
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
    const NodeLaunch nl = node_launch(g);
    k_prim<double><<<nl.grid, nl.block, 0, s>>>(g, ph, U, (double*)P, err);
    NA_CHECK(cudaGetLastError());
    if (params->scheme == CFD_HYBRID) {
        k_sensor<<<nl.grid, nl.block, 0, s>>>(g, ph, (const double*)P + 4 * N, cls);
        NA_CHECK(cudaGetLastError());
    }
    if (ph.viscous) {
        k_visc_flux<double><<<nl.grid, nl.block, 0, s>>>(g, ph, (const double*)P, (double*)Fv);
        NA_CHECK(cudaGetLastError());
    }
    SweepArgs A{};
    A.g = g;
    A.ph = ph;
    A.P = P;
    A.cls = params->scheme == CFD_HYBRID ? cls : nullptr;
    A.Fv = ph.viscous ? Fv : nullptr;
    A.R = R;
    A.Lout = dUdt;
    A.rk_b = 1.0;
    A.seg_len = 128;
    {
        const int lo = g.per[0] ? 0 : 1, hi = g.per[0] ? g.nx : g.nx - 1;
        const int nb = g.nx <= 32 ? 32 : (g.nx <= 64 ? 64 : 128);
        dim3 gr((hi - lo + nb - 1) / nb, g.ny, g.nz);
        if (nb == 32) k_sweep_x<double, 32, EP_STORE><<<gr, 32, 0, s>>>(A);
        else if (nb == 64) k_sweep_x<double, 64, EP_STORE><<<gr, 64, 0, s>>>(A);
        else k_sweep_x<double, 128, EP_STORE><<<gr, 128, 0, s>>>(A);
        NA_CHECK(cudaGetLastError());
    }
    const size_t smem = 4 * 80 * 32 * sizeof(double);
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
