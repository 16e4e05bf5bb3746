// cfd_kernels.cuh -- sm_103a kernels of the OpenCFD-SCU stage right-hand side
// (arXiv:2209.15333, Sections 2.1-2.4).
//
// Data layout in HBM (structure of arrays, i fastest, N = nx*ny*nz):
//   U, Un        [5][N]  double  conserved state (stage / step start)
//   P            [7][N]  real    rho, u, v, w, p, T, c
//   cls          [N]     uint8   sensor class (0 UD7, 1 WENO7, 2 WENO5)
//   Fv           [12][N] real    viscous fluxes at nodes, [4*d + row]
//   R            [5][N]  real    accumulated -sum delta fhat + sum D Fv
//   met          [31][M] double  metrics per metric point (M = N, nx*ny or 1):
//                                0-8 raw (xi_x..zeta_z), 9 J, 10-18 alpha = raw/J,
//                                19-21 sigma_d = |alpha_d|, 22-30 k_d = alpha_d/sigma_d
//   metf         [31][M] float   the same metrics rounded once, read by the FP32 kernels
#pragma once
#include <cstdint>
#include <type_traits>

#include <cuda.h>  // CUtensorMap (tensor-memory-accelerator descriptors); no driver calls here

#include "weno_coeffs.cuh"

namespace cfdk {

enum { M_RAW = 0, M_J = 9, M_ALPHA = 10, M_SIG = 19, M_K = 22, M_COUNT = 31 };

struct Geo {
    int nx, ny, nz;
    long long N;
    int per[3];
    int bc_lo[3], bc_hi[3];
    int mlayout;          // 0 3-D, 1 2-D, 2 uniform
    int diag;             // 1: every metric matrix is diagonal (uniform Cartesian box)
    // on such a box, a periodic direction d (gfold[d]) takes its Cartesian
    // derivative in the FP64 form from the central stencil with the metric
    // folded into the coefficients: gsc[d][k] = c_k d_x
    int gfold[3];
    double gsc[3][4];
    long long M;          // metric points
    const double* met;    // [31][M]
    const float* metf;    // [31][M] float mirror (FP32 kernels)
};

struct Phys {
    double gamma, gm1, inv_gm1, Ma, gMa2, inv2g, invMa;
    double invRe, kcoef;  // 1/Re, 1/((gamma-1) Ma^2 Pr Re)
    double Tw;
    int viscous, visc_law;
    double omega, suth_s;  // power exponent, S/T_ref
    // the power law's tables (see power_law; null: exp(omega log T)) and the
    // binomial coefficients C(omega, j) of its series
    const double* powtab;
    const float* powtabf;
    double pc[6];
    float pcf[3];
    int scheme;            // 0 UD7, 1 WENO5, 2 WENO7, 3 HYBRID
    int charrec;           // WENO faces reconstruct characteristic fields (Sec. 2.2.2)
    double th1, th2, eps;
    int vorder;
    // the constants rounded once to float, for the FP32 kernels (no
    // double-to-float conversion in the loops: it runs on the FP64 pipe)
    float gm1f, inv_gm1f, inv2gf, invRef, kcoeff, omegaf, suth_sf, th1f, th2f, epsf, gMa2f, invMaf, gammaf;
};

template <class R>
__device__ __forceinline__ R pk(double d, float f);
template <>
__device__ __forceinline__ double pk<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pk<float>(double, float f) { return f; }

// a * b + c with one rounding.  The stencil arithmetic shared by the kernel
// families (tiles, walks, streams, ensembles) is written with explicit fused
// multiply-adds in a fixed order: left to the compiler, a sum of two products
// may be contracted either way, differently in different kernels, and the
// families would no longer give the same bits.
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }

struct BCData {
    const double* inflow;  // [5][ny] or null
    double amp, x0, x1, omega, Lz;
    int m;
    const double* wall_x;  // [nx]
    const double* wall_z;  // [nz]
};

// periodic wrap of a line position m into [0, n): one period either way
// (selects, no loop) covers the stencil offsets of every line longer than
// them; only a position more than one period out (a periodic line shorter
// than the stencil) takes the integer division
__device__ __forceinline__ int wrapi(int m, int n)
{
    const int r = m < 0 ? m + n : (m >= n ? m - n : m);
    if ((unsigned)r < (unsigned)n) return r;
    const int q = m % n;
    return q < 0 ? q + n : q;
}

// a request of the 128-byte line holding p into L2 (no register, no wait)
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ long long midx(const Geo& g, int i, int j, long long n)
{
    return g.mlayout == 0 ? n : (g.mlayout == 1 ? (long long)i + (long long)g.nx * j : 0LL);
}

// Index-bounds checks of the bounds-checked build (CFD_BOUNDS_CHECK): an
// index outside [0, n) sets the flag 2 (bit 1) of the error word and the access is
// skipped; the normal build compiles the check away.
#ifdef CFD_BOUNDS_CHECK
__device__ __forceinline__ bool in_range(int* err, long long i, long long n)
{
    if (i >= 0 && i < n) return true;
    atomicOr(err, 2);
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_range(int*, long long, long long) { return true; }
#endif

__device__ __forceinline__ double metv(const Geo& g, int e, long long mi)
{
    return __ldg(g.met + (long long)e * g.M + mi);
}

template <class R>
__device__ __forceinline__ R metr(const Geo& g, int e, long long mi);
template <>
__device__ __forceinline__ double metr<double>(const Geo& g, int e, long long mi)
{
    return __ldg(g.met + (long long)e * g.M + mi);
}
template <>
__device__ __forceinline__ float metr<float>(const Geo& g, int e, long long mi)
{
    return __ldg(g.metf + (long long)e * g.M + mi);
}

// node (i, j, k) of a node-parallel kernel on a (x-chunks, ny, nz) grid of
// (virtual) blocks vb; the body that follows runs only when i < nx
// Node kernels: vb = (x segment, j, k) with x on threads, or (FLAT) vb.x
// counts runs of blockDim.x consecutive nodes of the flattened grid (N < 2^31;
// used by the ensemble, whose blocks can be narrower than a CTA).
#define NODE_IJK_SEL(g, FLAT)                                                                         \
    int i, j, k;                                                                                      \
    long long n;                                                                                      \
    bool node_ok_;                                                                                    \
    if constexpr (FLAT) {                                                                             \
        const unsigned t_ = vb.x * blockDim.x + threadIdx.x;                                          \
        const unsigned r_ = t_ / (unsigned)(g).nx;                                                    \
        i = (int)(t_ - r_ * (unsigned)(g).nx);                                                        \
        j = (int)(r_ % (unsigned)(g).ny);                                                             \
        k = (int)(r_ / (unsigned)(g).ny);                                                             \
        n = (long long)t_;                                                                            \
        node_ok_ = n < (g).N;                                                                         \
    } else {                                                                                          \
        i = vb.x * blockDim.x + threadIdx.x;                                                          \
        j = vb.y;                                                                                     \
        k = vb.z;                                                                                     \
        n = (long long)i + (long long)(g).nx * ((long long)j + (long long)(g).ny * k);                \
        node_ok_ = i < (g).nx;                                                                        \
    }                                                                                                 \
    if (node_ok_)
#define NODE_IJK(g) NODE_IJK_SEL(g, false)

__device__ __forceinline__ bool is_bnd(const Geo& g, int i, int j, int k)
{
    return (!g.per[0] && (i == 0 || i == g.nx - 1)) || (!g.per[1] && (j == 0 || j == g.ny - 1)) ||
           (!g.per[2] && (k == 0 || k == g.nz - 1));
}

// ---------------------------------------------------------------------------
// metric set-up: derived quantities per metric point (Eq. 19, 22, 27)
// ---------------------------------------------------------------------------
__global__ void k_metric_float(const double* met, float* metf, long long count)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        metf[t] = (float)met[t];
}

__global__ void k_metric_derive(double* met, long long M)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < M;
         t += (long long)gridDim.x * blockDim.x) {
        double J = met[M_J * M + t];
        for (int d = 0; d < 3; ++d) {
            double a[3];
            for (int e = 0; e < 3; ++e) {
                a[e] = met[(3 * d + e) * M + t] / J;
                met[(M_ALPHA + 3 * d + e) * M + t] = a[e];
            }
            double s = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            met[(M_SIG + d) * M + t] = s;
            for (int e = 0; e < 3; ++e) met[(M_K + 3 * d + e) * M + t] = a[e] / s;
        }
    }
}

// Everything a kernel of one stage needs about one block: geometry, gas,
// buffers and the RK3 epilogue.  Single-block launches pass it by value;
// batched launches read one per block from a device table.
struct SweepArgs {
    Geo g;
    Phys ph;
    void* P;               // [7][N] real primitives
    const uint8_t* cls;    // [N] classes read by the sweeps (null unless hybrid)
    uint8_t* cls_io;       // [N] classes written by the sensor / read by the mixed recovery
    void* Fv;              // [12][N] real or null (inviscid)
    void* R;               // [5][N] real accumulator
    int* err;              // non-physical flag
    const double* U;       // stage state  U^(k)
    const double* Un;      // step state   U^n
    double* Uout;          // RK output (may alias U or Un)
    double* Lout;          // L(U) output (rhs mode) or null
    const double* dt;      // device scalar
    double rk_a, rk_b;     // U_out = a Un + b (U + dt L)
    int seg_len;           // streaming segment length
};

// ---------------------------------------------------------------------------
// primitive recovery (Eq. 5, 8, 16, 17): one reciprocal of rho per node.  On
// GB300 every FP64 operation takes a slot of a narrow pipe (two per clock and
// SM), so the checks of a non-physical state run on the bit patterns in the
// integer pipe: rho and p positive and finite, |u|, |v|, |w| and T below 1e300.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool positive_finite(double x)
{
    // positive finite doubles are the bit patterns 1 .. 0x7FEFFFFFFFFFFFFF
    return (unsigned long long)__double_as_longlong(x) - 1ull < 0x7FEFFFFFFFFFFFFFull;
}
__device__ __forceinline__ bool below_1e300(double x)
{
    // |x| < 1e300 (false for NaN and infinities)
    return ((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) <
           (unsigned long long)__double_as_longlong(1e300);
}

// ---------------------------------------------------------------------------
// binary64 <-> binary32 format conversions on the integer pipe (IEEE 754
// field layouts: 1 sign, 11/8 exponent bits biased by 1023/127, 52/23
// fraction bits).  A hardware cvt between the two formats takes a slot of
// the narrow FP64 pipe; these take a handful of integer operations and give
// the same bits (checked against the hardware over every float and a
// structured sweep of doubles by cfd_check_conversions).
// ---------------------------------------------------------------------------
// float -> double, exact for every input (NaN stays NaN)
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned b = __float_as_uint(f), a = b & 0x7fffffffu;
    unsigned hi, lo = b << 29;                         // the low 3 fraction bits
    if (a - 0x00800000u < 0x7f000000u) {               // normal: exponent + (1023 - 127)
        hi = (a >> 3) + (896u << 20);
    } else if (a >= 0x7f800000u) {                     // infinity, NaN
        hi = (a >> 3) | 0x7ff00000u;
    } else if (a == 0u) {
        hi = 0u;
    } else {                                           // subnormal: normalise the fraction
        const unsigned sh = (unsigned)__clz((int)a) - 8u, m = a << sh;
        hi = ((m & 0x7fffffu) >> 3) + ((897u - sh) << 20);
        lo = m << 29;
    }
    return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// double -> float, round to nearest even.  ok is true, and the result the
// correctly rounded one, for zero and for every x whose float is normal or
// overflows by rounding (2^-126 <= |x| < 2^128); elsewhere (subnormal
// results, |x| >= 2^128, infinities, NaN) ok is false.
__device__ __forceinline__ float d2f_rn_int(double x, bool& ok)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned ah = hi & 0x7fffffffu;
    const unsigned t = __funnelshift_l(lo, ah - (896u << 20), 3);  // rebiased, fraction cut to 23 bits
    const unsigned r = lo & 0x1fffffffu;                            // the 29 fraction bits cut off
    const unsigned f = t + ((r + 0x0fffffffu + (t & 1u)) >> 29);   // half to even; may carry into the exponent
    const bool zero = (ah | lo) == 0u;
    ok = ah - (897u << 20) < (254u << 20) || zero;
    return __uint_as_float((hi & 0x80000000u) | (zero ? 0u : f));
}

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_exact(x); }

template <class RT, bool FLAT = false>
__device__ __forceinline__ void prim_body(const SweepArgs& A, uint3 vb)
{
    const Geo& g = A.g;
    const Phys& ph = A.ph;
    const double* __restrict__ U = A.U;
    RT* __restrict__ P = (RT*)A.P;
    int* err = A.err;
    const long long N = g.N;
    NODE_IJK_SEL(g, FLAT)
    {
        const double rho = U[n];
        const double ri = 1.0 / rho;
        const double u = U[N + n] * ri;
        const double v = U[2 * N + n] * ri;
        const double w = U[3 * N + n] * ri;
        const double q2 = mad(w, w, mad(v, v, u * u));
        const double p = ph.gm1 * mad(-0.5 * rho, q2, U[4 * N + n]);
        const double T = ph.gMa2 * p * ri;
        const double c = sqrt(T) * ph.invMa;
        if (!positive_finite(rho) || !positive_finite(p) || !below_1e300(T) || !below_1e300(u) ||
            !below_1e300(v) || !below_1e300(w))
            *err = 1;
        P[n] = (RT)rho;
        P[N + n] = (RT)u;
        P[2 * N + n] = (RT)v;
        P[3 * N + n] = (RT)w;
        P[4 * N + n] = (RT)p;
        P[5 * N + n] = (RT)T;
        P[6 * N + n] = (RT)c;
    }
}

// Mixed precision: primitives in FP32 arithmetic, except within 4 nodes of a
// wall and at nodes whose previous sensor class is not UD7 (shocks), where the
// recovery runs in FP64 (catastrophic cancellation in E - rho|u|^2/2 is worst
// there); stored as float in both cases.  The FP32 recovery rounds the
// conserved variables to float on the integer pipe; a node with one of them
// outside float's normal range (nonzero below 2^-126 or at least 2^128) takes
// the FP64 recovery too.
__device__ __forceinline__ bool near_wall(const Geo& g, int i, int j, int k)
{
    const int pos[3] = {i, j, k};
    const int nd[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (g.bc_lo[d] == 1 && pos[d] < 4) return true;
        if (g.bc_hi[d] == 1 && pos[d] > nd[d] - 5) return true;
    }
    return false;
}

template <bool FLAT = false>
__device__ __forceinline__ void prim_mixed_body(const SweepArgs& A, uint3 vb)
{
    const Geo& g = A.g;
    const Phys& ph = A.ph;
    const double* __restrict__ U = A.U;
    float* __restrict__ P = (float*)A.P;
    const uint8_t* __restrict__ cls_prev = A.cls_io;
    int* err = A.err;
    const long long N = g.N;
    NODE_IJK_SEL(g, FLAT)
    {
        float rho, u, v, w, p, T, c;
        bool ok[5];
        float q[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) q[e] = d2f_rn_int(U[e * N + n], ok[e]);
        if (cls_prev[n] != 0 || near_wall(g, i, j, k) || !(ok[0] && ok[1] && ok[2] && ok[3] && ok[4])) {
            double rd = U[n];
            double ri = 1.0 / rd;
            double ud = U[N + n] * ri, vd = U[2 * N + n] * ri, wd = U[3 * N + n] * ri;
            double pd = ph.gm1 * mad(-0.5 * rd, mad(wd, wd, mad(vd, vd, ud * ud)), U[4 * N + n]);
            double Td = ph.gMa2 * pd * ri;
            rho = (float)rd; u = (float)ud; v = (float)vd; w = (float)wd; p = (float)pd; T = (float)Td;
            c = sqrtf(T) * ph.invMaf;
        } else {
            rho = q[0];
            float ri = 1.0f / rho;
            u = q[1] * ri;
            v = q[2] * ri;
            w = q[3] * ri;
            p = ph.gm1f * mad(-0.5f * rho, mad(w, w, mad(v, v, u * u)), q[4]);
            T = ph.gMa2f * p * ri;
            c = sqrtf(T) * ph.invMaf;
        }
        if (!(rho > 0.0f) || !(p > 0.0f) || !(T < 1e30f) || !(fabsf(u) + fabsf(v) + fabsf(w) < 1e30f)) *err = 1;
        P[n] = rho;
        P[N + n] = u;
        P[2 * N + n] = v;
        P[3 * N + n] = w;
        P[4 * N + n] = p;
        P[5 * N + n] = T;
        P[6 * N + n] = c;
    }
}

// ---------------------------------------------------------------------------
// modified Jameson sensor (Eq. 42-43) in FP64 without a division: with
// phi_d = a_d/b_d (a_d = |p_{m-1} - 2 p_m + p_{m+1}|, b_d = p_{m-1} + 2 p_m +
// p_{m+1} > 0), theta <= theta_k is decided as
//   a_0 b_1 b_2 + a_1 b_0 b_2 + a_2 b_0 b_1 <= theta_k b_0 b_1 b_2,
// the same inequality multiplied by the positive common denominator (the
// decision can differ from a summed-quotient evaluation only where theta lies
// within a few units of rounding of a threshold).  Both sides are
// non-negative, so they compare as integers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool nonneg_le(double a, double b)
{
    return __double_as_longlong(a) <= __double_as_longlong(b);
}

template <bool FLAT = false>
__device__ __forceinline__ void sensor_body(const SweepArgs& A, uint3 vb)
{
    const Geo& g = A.g;
    const Phys& ph = A.ph;
    const double* __restrict__ p = (const double*)A.P + 4 * g.N;
    uint8_t* __restrict__ cls = A.cls_io;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    NODE_IJK_SEL(g, FLAT)
    {
        const double p0 = p[n];
        const double p2 = p0 + p0;
        double a[3], b[3];
        const int pos[3] = {i, j, k};
        const int nd[3] = {nx, ny, nz};
        const long long st[3] = {1, nx, (long long)nx * ny};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int m = pos[d];
            if (!g.per[d] && (m == 0 || m == nd[d] - 1)) {
                a[d] = 0.0;  // phi_d = 0 at a non-periodic boundary node (reading R4)
                b[d] = 1.0;
                continue;
            }
            const double pm = p[n + (long long)(wrapi(m - 1, nd[d]) - m) * st[d]];
            const double pp = p[n + (long long)(wrapi(m + 1, nd[d]) - m) * st[d]];
            a[d] = fabs((p2 - pm) - pp);
            b[d] = (pm + p2) + pp;
        }
        const double b12 = b[1] * b[2];
        const double num = mad(a[2], b[0] * b[1], mad(a[1], b[0] * b[2], a[0] * b12));
        const double den = b[0] * b12;
        cls[n] = nonneg_le(num, ph.th1 * den) ? 0 : (nonneg_le(num, ph.th2 * den) ? 1 : 2);
    }
}

// the same sensor in FP32 arithmetic on FP32 pressures (mixed precision)
template <bool FLAT = false>
__device__ __forceinline__ void sensor32_body(const SweepArgs& A, uint3 vb)
{
    const Geo& g = A.g;
    const Phys& ph = A.ph;
    const float* __restrict__ p = (const float*)A.P + 4 * g.N;
    uint8_t* __restrict__ cls = A.cls_io;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const float th1 = ph.th1f, th2 = ph.th2f;
    NODE_IJK_SEL(g, FLAT)
    {
        float p0 = p[n];
        const int pos[3] = {i, j, k};
        const int nd[3] = {nx, ny, nz};
        const long long st[3] = {1, nx, (long long)nx * ny};
        float th = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int m = pos[d];
            if (!g.per[d] && (m == 0 || m == nd[d] - 1)) continue;
            float pm = p[n + (long long)(wrapi(m - 1, nd[d]) - m) * st[d]];
            float pp = p[n + (long long)(wrapi(m + 1, nd[d]) - m) * st[d]];
            const float p2 = p0 + p0;
            th += fabsf((p2 - pm) - pp) / ((pm + p2) + pp);
        }
        cls[n] = th <= th1 ? 0 : (th <= th2 ? 1 : 2);
    }
}

// ---------------------------------------------------------------------------
// learned shock sensor: 42 normalised stencil differences of p and rho ->
// 32 -> 32 -> 3 MLP (BF16 weights, FP32 accumulation on the tensor cores
// with mma.sync m16n8k16), falling back to the plain sensor (Eq. 42-43) when
// the largest softmax probability is below conf_min or an input is not finite.
// Features, for each direction d and field q in (p, rho), over the line
// positions m-3..m+3 (periodic lines wrap, others clamp at the ends):
//   (q_{m+t+1} - q_{m+t}) / q_m for t = -3..2, and
//   (q_{m-1} - 2 q_m + q_{m+1}) / (q_{m-1} + 2 q_m + q_{m+1});
// feature index (2 d + field) * 7 + t.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// mbarrier and tensor-memory-accelerator copies (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit)
{
    for (unsigned it = 0; it < limit; ++it) {
        if (mbar_test(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

constexpr unsigned TW_WAIT_LIMIT = 1u << 22;  // polls of a bounded mbarrier wait (about 0.3 s)

enum { MLP_IN = 42, MLP_H = 32, MLP_OUT = 3, MLP_KP = 48, MLP_NP = 8 };

struct MlpArgs {
    const uint16_t* w1;  // [32][48] bf16, in padded with zeros
    const uint16_t* w2;  // [32][32] bf16
    const uint16_t* w3;  // [8][32] bf16, rows 3..7 zero
    const float* b1;     // [32]
    const float* b2;     // [32]
    const float* b3;     // [8]
    float conf_min;
    unsigned long long* fallbacks;  // count of nodes that fell back to the plain sensor
};

// the seven features of one field along one direction from the values at
// line positions m-3 .. m+3 (one routine for every kernel that builds them,
// so that they agree bit for bit); inv = 1 / v[3], the node's own value,
// which its three lines share
__device__ __forceinline__ void mlp_feature_line_inv(const float v[7], float inv, float* o)
{
#pragma unroll
    for (int t = 0; t < 6; ++t) o[t] = (v[t + 1] - v[t]) * inv;
    const float v2 = v[3] + v[3];
    // a ratio in [-1, 1] for positive p and rho: the fast division's few
    // units of rounding are far below the bf16 rounding of the inputs
    o[6] = __fdividef((v[2] - v2) + v[4], (v[2] + v2) + v[4]);
}
__device__ __forceinline__ void mlp_feature_line(const float v[7], float* o)
{
    mlp_feature_line_inv(v, 1.0f / v[3], o);
}

// line position m + t (t = -3..3) with periodic wrap or clamping at the ends
__device__ __forceinline__ int mlp_pos(int m, int t, int n, int per)
{
    int mm = m + t;
    if (per) return wrapi(mm, n);
    return mm < 0 ? 0 : (mm >= n ? n - 1 : mm);
}

template <class RT>
__device__ __forceinline__ void mlp_features(const SweepArgs& A, int i, int j, int k, long long n, float f[MLP_IN])
{
    const Geo& g = A.g;
    const RT* P = (const RT*)A.P;
    const long long N = g.N;
    const int pos[3] = {i, j, k};
    const int nd[3] = {g.nx, g.ny, g.nz};
    const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int m = pos[d];
        long long off[7];
#pragma unroll
        for (int t = 0; t < 7; ++t) off[t] = (long long)(mlp_pos(m, t - 3, nd[d], g.per[d]) - m) * st[d];
#pragma unroll
        for (int fld = 0; fld < 2; ++fld) {
            const RT* q = P + (fld == 0 ? 4 * N : 0) + n;
            float v[7];
#pragma unroll
            for (int t = 0; t < 7; ++t) v[t] = (float)q[off[t]];
            mlp_feature_line(v, f + (2 * d + fld) * 7);
        }
    }
}

// two floats to a pair of bf16 (round to nearest even), lo in the low half
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// plain-sensor class of one node in the kernel's precision (the fallback)
template <class RT>
__device__ __forceinline__ int plain_class(const SweepArgs& A, int i, int j, int k, long long n)
{
    const Geo& g = A.g;
    const RT* p = (const RT*)A.P + 4 * g.N;
    const int pos[3] = {i, j, k};
    const int nd[3] = {g.nx, g.ny, g.nz};
    const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
    RT th = (RT)0;
    for (int d = 0; d < 3; ++d) {
        const int m = pos[d];
        if (!g.per[d] && (m == 0 || m == nd[d] - 1)) continue;
        const RT pm = p[n + (long long)(wrapi(m - 1, nd[d]) - m) * st[d]];
        const RT pp = p[n + (long long)(wrapi(m + 1, nd[d]) - m) * st[d]];
        const RT p0 = p[n];
        th += fabs(-pm + (RT)2 * p0 - pp) / (pm + (RT)2 * p0 + pp);
    }
    return th <= (RT)A.ph.th1 ? 0 : (th <= (RT)A.ph.th2 ? 1 : 2);
}

constexpr int MLP_ROW = 56;  // bf16 row stride of the feature tile (conflict-free fragment loads)

// the network's weights and biases in shared memory (bf16 rows padded for
// conflict-free B-fragment loads)
struct MlpWeightsSmem {
    uint16_t sw1[32 * MLP_ROW];
    uint16_t sw2[32 * 40];
    uint16_t sw3[8 * 40];
    float sb[32 + 32 + 8];
};

__device__ __forceinline__ void mlp_stage_weights(MlpWeightsSmem& S, const MlpArgs& W)
{
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < 32 * MLP_KP; e += nt) S.sw1[(e / MLP_KP) * MLP_ROW + e % MLP_KP] = W.w1[e];
    for (int e = t; e < 32 * 32; e += nt) S.sw2[(e / 32) * 40 + e % 32] = W.w2[e];
    for (int e = t; e < 8 * 32; e += nt) S.sw3[(e / 32) * 40 + e % 32] = W.w3[e];
    for (int e = t; e < 72; e += nt) S.sb[e] = e < 32 ? W.b1[e] : (e < 64 ? W.b2[e - 32] : W.b3[e - 64]);
}

// four (two) 8 x 8 bf16 matrices from shared memory in the mma fragment
// layout: lane L gives the address of row L mod 8 of matrix L / 8
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// ReLU on a packed pair of bf16 (max with +0; a NaN gives 0)
__device__ __forceinline__ uint32_t relu_bf16x2(uint32_t x)
{
    uint32_t r;
    asm("max.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(0u));
    return r;
}

// accumulator fragments of a [16 x 32] layer output, biases as the initial
// value, to bf16 pairs with ReLU: the A fragments of the next layer
__device__ __forceinline__ void mlp_hidden_init(float h[4][4], const float* bias)
{
    const int tig = threadIdx.x & 3;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float2 b = *reinterpret_cast<const float2*>(bias + nt * 8 + tig * 2);
        h[nt][0] = b.x, h[nt][1] = b.y, h[nt][2] = b.x, h[nt][3] = b.y;
    }
}
__device__ __forceinline__ void mlp_hidden_pack(const float h[4][4], uint32_t a[2][4])
{
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        a[nt >> 1][(nt & 1) * 2 + 0] = relu_bf16x2(pack_bf16x2(h[nt][0], h[nt][1]));
        a[nt >> 1][(nt & 1) * 2 + 1] = relu_bf16x2(pack_bf16x2(h[nt][2], h[nt][3]));
    }
}

// The three layers on the tensor cores for the 32 rows of one warp's feature
// tile sx (rows 0..31, stride MLP_ROW); every lane gets the class of row
// `lane`, -1 where the top softmax probability is below conf_min (or not
// finite).  Fragments come from shared memory by ldmatrix, biases enter as
// the accumulators' initial values.  Warp-synchronous: the caller orders the
// rows' writes before it (__syncwarp) and any rewrite after it.
__device__ __forceinline__ int mlp_classify_warp(const uint16_t* sx, const MlpWeightsSmem& S, float conf_min)
{
    const int lane = threadIdx.x & 31;
    const int tig = lane & 3;
    // ldmatrix row addresses: A (rows lane mod 16, k half lane / 16); B pairs
    // of n-tiles (n row lane mod 8 + 8 (lane / 16), k half (lane / 8) mod 2);
    // layer 3 (n row lane mod 8, k eighth lane / 8)
    const uint16_t* arow = sx + (lane & 15) * MLP_ROW + (lane >> 4) * 8;
    const int bn = (lane & 7) + ((lane >> 4) << 3), bk = ((lane >> 3) & 1) * 8;
    const uint16_t* b1row = S.sw1 + bn * MLP_ROW + bk;
    const uint16_t* b2row = S.sw2 + bn * 40 + bk;
    // row L = 16 mt + 8 half + g: its logits 0, 1 sit in lg[2 half], lg[2 half + 1]
    // of lane 4 g after m-tile mt, logit 2 in lg[2 half] of lane 4 g + 1
    const int g4 = (lane & 7) * 4, my_mt = lane >> 4, half = (lane >> 3) & 1;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        // layer 1: [16 x 48] x [48 x 32]
        float h1[4][4];
        mlp_hidden_init(h1, S.sb);
#pragma unroll
        for (int ks = 0; ks < 3; ++ks) {
            uint32_t a[4];
            ldsm_x4(a, arow + mt * 16 * MLP_ROW + ks * 16);
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                uint32_t b[4];
                ldsm_x4(b, b1row + np * 16 * MLP_ROW + ks * 16);
                mma_bf16_16816(h1[2 * np], a, b);
                mma_bf16_16816(h1[2 * np + 1], a, b + 2);
            }
        }
        uint32_t a2[2][4];
        mlp_hidden_pack(h1, a2);
        // layer 2: [16 x 32] x [32 x 32]
        float h2[4][4];
        mlp_hidden_init(h2, S.sb + 32);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                uint32_t b[4];
                ldsm_x4(b, b2row + np * 16 * 40 + ks * 16);
                mma_bf16_16816(h2[2 * np], a2[ks], b);
                mma_bf16_16816(h2[2 * np + 1], a2[ks], b + 2);
            }
        }
        uint32_t a3[2][4];
        mlp_hidden_pack(h2, a3);
        // layer 3: [16 x 32] x [32 x 8] (3 logits used)
        const float2 b3 = *reinterpret_cast<const float2*>(S.sb + 64 + tig * 2);
        float lg[4] = {b3.x, b3.y, b3.x, b3.y};
        uint32_t b[4];
        ldsm_x4(b, S.sw3 + (lane & 7) * 40 + (lane >> 3) * 8);
        mma_bf16_16816(lg, a3[0], b);
        mma_bf16_16816(lg, a3[1], b + 2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float x0 = __shfl_sync(0xffffffffu, lg[2 * h], g4);
            const float x1 = __shfl_sync(0xffffffffu, lg[2 * h + 1], g4);
            const float x2 = __shfl_sync(0xffffffffu, lg[2 * h], g4 + 1);
            if (mt == my_mt && h == half) c0 = x0, c1 = x1, c2 = x2;
        }
    }
    const float mx = fmaxf(c0, fmaxf(c1, c2));
    const float z = __expf(c0 - mx) + __expf(c1 - mx) + __expf(c2 - mx);
    const int arg = c0 >= c1 ? (c0 >= c2 ? 0 : 2) : (c1 >= c2 ? 1 : 2);
    return (1.0f / z >= conf_min && isfinite(z)) ? arg : -1;
}

// Learned sensor, walking form.  A CTA of 8 warps owns a 32 x 8 (x, y) column
// of nodes and walks zeta over `tz` planes.  p and rho of each plane, with a
// 3-node x/y halo (38 x 14 values, periodic lines wrapped, others clamped as
// the features define), are loaded once into a ring of 8 planes in shared
// memory; the next plane's loads are issued before the current plane's
// features and stored into the ring after them.  The features of
// plane z come from the ring: x and y lines from plane z, zeta lines from
// planes z-3 .. z+3.  Warp w holds the nodes of y-row w and classifies its
// own 32 feature rows, so the only CTA barrier per plane orders the ring:
// plane z+4 overwrites plane z-4, whose last reader was plane z-1.
constexpr int MW_X = 32 + 6, MW_Y = 8 + 6, MW_PL = MW_X * MW_Y;  // staged plane: 38 x 14
constexpr int MW_RING = 8;

struct MlpWalkSmem {
    float ring[MW_RING][2][MW_PL];  // [plane mod 8][p, rho][hy * 38 + hx]
    uint16_t sx[256 * MLP_ROW];     // bf16 feature rows, row = warp * 32 + lane
    MlpWeightsSmem w;
};

// ---------------------------------------------------------------------------
// The same three layers on the fifth-generation tensor cores (tcgen05, inline
// PTX).  A CTA's 256 feature rows (its 32 x 8 nodes of one plane) form two
// M = 128 tiles; one thread issues the MMAs of a layer (bf16 operands from
// shared memory, FP32 accumulators in tensor memory) and commits them to an
// mbarrier; every warp then reads its own 32 rows back (tcgen05.ld: warp w
// reaches lanes 32 (w mod 4) ..), adds the biases, applies ReLU and writes the
// next layer's bf16 operand.  Operands are K-major without swizzle: "core
// matrices" of 8 rows x 16 bytes stored contiguously, the K-adjacent ones 128
// bytes apart (leading byte offset), the 8-row groups KC x 128 bytes apart
// (stride byte offset), KC = K / 8.  Biases are added to the accumulators
// after the products (the warp-level form starts from them), so the two
// forms can differ in the last bits of a logit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor (start address, leading and stride byte
// offsets in 16-byte units, descriptor version 1, no swizzle)
__device__ __forceinline__ uint64_t tc_smem_desc(const void* p, uint32_t lbo, uint32_t sbo)
{
    const uint64_t a = smem_u32(p);
    return ((a >> 4) & 0x3FFFull) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16
// A and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24
constexpr uint32_t tc_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}
// arrive on the mbarrier once every MMA this thread issued has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 columns of this thread's tensor-memory lane (load and its wait in one
// statement, so that no use of v can be scheduled before the wait)
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, float (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_x4(uint32_t taddr, float (&v)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(taddr)
                 : "memory");
}
// tensor-memory columns of one CTA (a power of two >= 32), allocated by warp 0
constexpr uint32_t MLP_TMEM_COLS = 64;
__device__ __forceinline__ void tmem_alloc_warp(uint32_t* slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
                 "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::"r"(smem_u32(slot)),
                 "r"(MLP_TMEM_COLS)
                 : "memory");
}
__device__ __forceinline__ void tmem_dealloc_warp(uint32_t base)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(MLP_TMEM_COLS) : "memory");
}

// shared memory of the tensor-core walk: the p / rho ring of the warp-level
// form, the operand tile and the weights, all in the core-matrix layout.  The
// operand tile holds the features (K = 48) and, once a layer's MMAs have
// completed, the hidden activations that feed the next (K = 32): 65 KB, three
// CTAs per SM
struct MlpTcSmem {
    float ring[MW_RING][2][MW_PL];
    alignas(16) uint16_t ax[2 * 16 * 6 * 64];  // [tile][row group][K chunk][8 x 8]
    alignas(16) uint16_t w1[4 * 6 * 64];       // [n group][K chunk][8 x 8], N = 32, K = 48
    alignas(16) uint16_t w2[4 * 4 * 64];       // N = 32, K = 32
    alignas(16) uint16_t w3[2 * 4 * 64];       // N = 16 (rows 3..15 zero), K = 32
    float b[32 + 32 + 8];
    uint64_t bar;
    uint32_t tmem;
};
// element (row, k) of a core-matrix tile with KC chunks of 8 along K
__device__ __forceinline__ int tc_off(int row, int k, int KC)
{
    return (((row >> 3) * KC + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// weights to shared memory, the mbarrier, and the CTA's tensor memory
__device__ __forceinline__ void mlp_tc_setup(MlpTcSmem& S, const MlpArgs& W)
{
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < 32 * MLP_KP; e += nt) S.w1[tc_off(e / MLP_KP, e % MLP_KP, 6)] = W.w1[e];
    for (int e = t; e < 32 * 32; e += nt) S.w2[tc_off(e / 32, e % 32, 4)] = W.w2[e];
    for (int e = t; e < 16 * 32; e += nt) S.w3[tc_off(e / 32, e % 32, 4)] = e < 8 * 32 ? W.w3[e] : (uint16_t)0;
    for (int e = t; e < 72; e += nt) S.b[e] = e < 32 ? W.b1[e] : (e < 64 ? W.b2[e - 32] : W.b3[e - 64]);
    if (t == 0) {
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) tmem_alloc_warp(&S.tmem);
    fence_proxy_async_smem();  // the weights, for the tensor cores' reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
__device__ __forceinline__ void mlp_tc_teardown(MlpTcSmem& S)
{
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc_warp(S.tmem);
    }
}

// bias, ReLU and bf16 packing of one row's 32 accumulators into the hidden tile
__device__ __forceinline__ void mlp_tc_hidden(MlpTcSmem& S, const float (&v)[32], const float* bias, int tile, int rr)
{
    uint16_t* h = S.ax + tile * (16 * 4 * 64);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t q[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            q[e] = relu_bf16x2(pack_bf16x2(v[8 * c + 2 * e] + bias[8 * c + 2 * e], v[8 * c + 2 * e + 1] + bias[8 * c + 2 * e + 1]));
        *reinterpret_cast<uint4*>(h + tc_off(rr, 8 * c, 4)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
}

// one layer's MMAs for both row tiles (thread 0), committed to the mbarrier;
// then every thread waits for them (bounded; flag 16 of the error word if
// they did not complete)
template <int KC, int N>
__device__ __forceinline__ bool mlp_tc_layer(MlpTcSmem& S, const uint16_t* a, const uint16_t* b, uint32_t& phase,
                                             int* err)
{
    if (threadIdx.x == 0) {
        tc_fence_after();
        constexpr uint32_t idesc = tc_idesc_bf16(128, N);
#pragma unroll
        for (int tile = 0; tile < 2; ++tile)
#pragma unroll
            for (int ks = 0; ks < KC / 2; ++ks)
                tc_mma_bf16(S.tmem + (uint32_t)(tile * 32), tc_smem_desc(a + tile * (16 * KC * 64) + ks * 128, 128, KC * 128),
                            tc_smem_desc(b + ks * 128, 128, KC * 128), idesc, ks > 0);
        tc_commit(&S.bar);
    }
    const bool ok = mbar_wait_bounded(&S.bar, phase & 1u, TW_WAIT_LIMIT);
    ++phase;
    if (!ok && err) atomicOr(err, 16);
    tc_fence_after();
    return ok;
}

// the class of this thread's row (row = warp * 32 + lane of the feature tile
// S.ax, written by the caller); -1 where the top softmax probability is below
// conf_min, not finite, or a wait gave up.  Every thread of the CTA calls it.
__device__ __forceinline__ int mlp_classify_tc(MlpTcSmem& S, float conf_min, uint32_t& phase, int* err)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = w >> 2, rr = (w & 3) * 32 + lane;
    const uint32_t trow = S.tmem + ((uint32_t)((w & 3) * 32) << 16) + (uint32_t)(tile * 32);
    fence_proxy_async_smem();  // this thread's feature rows, for the tensor cores
    __syncthreads();
    bool ok = mlp_tc_layer<6, 32>(S, S.ax, S.w1, phase, err);
    float v[32];
    tmem_ld_x32(trow, v);
    mlp_tc_hidden(S, v, S.b, tile, rr);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    ok = mlp_tc_layer<4, 32>(S, S.ax, S.w2, phase, err) && ok;
    tmem_ld_x32(trow, v);
    // (the completed MMAs have read their operand: the tile is free)
    mlp_tc_hidden(S, v, S.b + 32, tile, rr);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    ok = mlp_tc_layer<4, 16>(S, S.ax, S.w3, phase, err) && ok;
    float lg[4];
    tmem_ld_x4(trow, lg);
    tc_fence_before();  // the next plane's MMAs overwrite these columns
    const float c0 = lg[0] + S.b[64], c1 = lg[1] + S.b[65], c2 = lg[2] + S.b[66];
    const float mx = fmaxf(c0, fmaxf(c1, c2));
    const float z = __expf(c0 - mx) + __expf(c1 - mx) + __expf(c2 - mx);
    const int arg = c0 >= c1 ? (c0 >= c2 ? 0 : 2) : (c1 >= c2 ? 1 : 2);
    return (ok && 1.0f / z >= conf_min && isfinite(z)) ? arg : -1;
}

// one column's walk (vb: column x, column y, zeta segment); the weights are
// staged before the call.  SM = MlpWalkSmem: each warp classifies its rows
// with mma.sync; SM = MlpTcSmem: the CTA classifies its 256 rows with tcgen05
// (phase: the CTA's count of completed mbarrier phases)
template <class RT, class SM>
__device__ __forceinline__ void sensor_mlp_col(const SweepArgs& A, const MlpArgs& W, SM& S, uint3 vb, int tz,
                                               uint32_t& phase)
{
    constexpr bool TC = std::is_same<SM, MlpTcSmem>::value;
    const Geo& g = A.g;
    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long N = g.N, plane = (long long)nx * ny;
    const RT* Pp = (const RT*)A.P + 4 * N;
    const RT* Pr = (const RT*)A.P;
    const int x0 = vb.x * 32, y0 = vb.y * 8;
    const int z0 = vb.z * tz, z1 = min(z0 + tz, nz);
    // the staged positions of this thread (t, t + 256, t + 512 of the 532)
    // and their offsets within a plane, the same for every plane
    int poff[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int e = t + 256 * r;
        const int hy = e / MW_X, hx = e - hy * MW_X;
        poff[r] = e < MW_PL ? mlp_pos(x0 - 3, hx, nx, g.per[0]) + nx * mlp_pos(y0 - 3, hy, ny, g.per[1]) : 0;
    }
    auto load_plane = [&](int z, float (&v)[3][2]) {
        const long long base = (long long)mlp_pos(z, 0, nz, g.per[2]) * plane;
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (t + 256 * r < MW_PL) {
                v[r][0] = (float)__ldg(Pp + base + poff[r]);
                v[r][1] = (float)__ldg(Pr + base + poff[r]);
            }
    };
    auto store_plane = [&](int z, const float (&v)[3][2]) {
        const int slot = z & (MW_RING - 1);
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (t + 256 * r < MW_PL) {
                S.ring[slot][0][t + 256 * r] = v[r][0];
                S.ring[slot][1][t + 256 * r] = v[r][1];
            }
    };
    // prologue: planes z0-3 .. z0+3
    for (int z = z0 - 3; z <= z0 + 3; ++z) {
        float v[3][2];
        load_plane(z, v);
        store_plane(z, v);
    }
    __syncthreads();
    const int i = x0 + tx, j = y0 + ty;
    const bool own = i < nx && j < ny;
    const int ctr = (ty + 3) * MW_X + tx + 3;  // the node in a staged plane
    // this thread's feature row: chunks of 8 features, 16 bytes each
    uint4* row;
    if constexpr (TC) {
        const int rr = (ty & 3) * 32 + tx;  // row within tile ty / 4
        row = reinterpret_cast<uint4*>(S.ax + (ty >> 2) * (16 * 6 * 64) + tc_off(rr, 0, 6));
    } else {
        row = reinterpret_cast<uint4*>(S.sx + (ty * 32 + tx) * MLP_ROW);
    }
    // consecutive chunks of a row: 16 bytes apart, or one core matrix (128 bytes)
    constexpr int CS = TC ? 8 : 1;
    for (int z = z0; z < z1; ++z) {
        // plane z+4 is read by the outputs up to z1-1 while z+4 <= z1+2
        const bool more = z + 4 <= z1 + 2;
        float nxt[3][2];
        if (more) load_plane(z + 4, nxt);
        // the 42 features in order (direction, field, position), packed to
        // bf16 pairs and stored 8 at a time as they are produced; one test of
        // finiteness for all (x * 0 is 0 for finite x, NaN otherwise)
        const float* c0 = S.ring[z & (MW_RING - 1)][0];
        const float inv[2] = {1.0f / c0[ctr], 1.0f / c0[MW_PL + ctr]};
        float zc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        uint32_t w[4];
        float lo = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int fld = 0; fld < 2; ++fld) {
                const float* c = c0 + fld * MW_PL;
                float v[7], o[7];
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    v[q] = d == 0 ? c[ctr + q - 3]
                                  : (d == 1 ? c[ctr + (q - 3) * MW_X]
                                            : S.ring[(z + q - 3) & (MW_RING - 1)][fld][ctr]);
                mlp_feature_line_inv(v, inv[fld], o);
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const int e = (2 * d + fld) * 7 + q;
                    zc[e & 3] = fmaf(o[q], 0.0f, zc[e & 3]);
                    if (e & 1) w[(e >> 1) & 3] = pack_bf16x2(lo, o[q]);
                    else lo = o[q];
                    if ((e & 7) == 7) row[(e >> 3) * CS] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        // features 42..47 are zero padding
        w[1] = pack_bf16x2(lo, 0.0f);
        row[5 * CS] = make_uint4(w[0], w[1], 0u, 0u);
        // plane z+4 takes the slot of plane z-4 (no reader since the last barrier)
        if (more) store_plane(z + 4, nxt);
        const bool bad = !own || !((zc[0] + zc[1]) + (zc[2] + zc[3]) == 0.0f);
        if (bad) {
#pragma unroll
            for (int q = 0; q < MLP_KP / 8; ++q) row[q * CS] = make_uint4(0u, 0u, 0u, 0u);
        }
        int cls;
        if constexpr (TC) {
            cls = mlp_classify_tc(S, W.conf_min, phase, A.err);
        } else {
            __syncwarp();
            cls = mlp_classify_warp(S.sx + ty * 32 * MLP_ROW, S.w, W.conf_min);
        }
        if (own) {
            const long long n = (long long)i + (long long)nx * ((long long)j + (long long)ny * z);
            int c = cls;
            if (c < 0 || bad) {
                c = plain_class<RT>(A, i, j, z, n);
                if (W.fallbacks) atomicAdd(W.fallbacks, 1ull);
            }
            A.cls_io[n] = (uint8_t)c;
        }
        __syncthreads();
    }
}

template <class RT>
__global__ void __launch_bounds__(256, 2) k_sensor_mlp(SweepArgs A, MlpArgs W, int tz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpWalkSmem& S = *reinterpret_cast<MlpWalkSmem*>(smem_raw);
    mlp_stage_weights(S.w, W);
    uint32_t phase = 0;
    sensor_mlp_col<RT>(A, W, S, blockIdx, tz, phase);
}
// the walk with the layers on tcgen05 (tensor memory held for the CTA's life)
template <class RT>
__global__ void __launch_bounds__(256, 3) k_sensor_mlp_tc(SweepArgs A, MlpArgs W, int tz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpTcSmem& S = *reinterpret_cast<MlpTcSmem*>(smem_raw);
    mlp_tc_setup(S, W);
    uint32_t phase = 0;
    sensor_mlp_col<RT>(A, W, S, blockIdx, tz, phase);
    mlp_tc_teardown(S);
}

// the 42 features of every node (for training data and tests), [42][N] float
template <class RT>
__global__ void k_mlp_features(SweepArgs A, float* out)
{
    const Geo& g = A.g;
    const uint3 vb = blockIdx;
    NODE_IJK(g)
    {
        float f[MLP_IN];
        mlp_features<RT>(A, i, j, k, n, f);
#pragma unroll
        for (int e = 0; e < MLP_IN; ++e) out[(long long)e * g.N + n] = f[e];
    }
}

// ---------------------------------------------------------------------------
// Steger-Warming split fluxes at one node (Eq. 20-30, Eq. 23 as corrected).
// With s = l4 + l5 and dl = l5 - l4 the corrected Eq. 23 reads
//   f0 = a (2(g-1) l1 + s),  f_i = u_i f0 + a c dl k_i,
//   f4 = a ((g-1) l1 |u|^2 + s H + c dl (u.k)),   a = rho/(2 g),
// with H = |u|^2/2 + c^2/(g-1) (the same algebra, fewer operations).
// ---------------------------------------------------------------------------
// positive and negative parts max(x, 0), min(x, 0) (Eq. 29); in FP64 on the
// sign bit in the integer pipe (the FP64 pipe is the bottleneck on GB300)
__device__ __forceinline__ double pos_part(double x)
{
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(b & ~(b >> 63));
}
__device__ __forceinline__ double neg_part(double x)
{
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(b & (b >> 63));
}
__device__ __forceinline__ float pos_part(float x) { return fmaxf(x, 0.0f); }
__device__ __forceinline__ float neg_part(float x) { return fminf(x, 0.0f); }

template <class R>
// axis = 0, 1, 2: k is that unit vector (the directions of a uniform
// diagonal box), whose zero components cost nothing; -1: any k.  The FP64
// form uses the axis form on such boxes (the FP64 pipe bounds it); in FP32
// the second inlined copy costs more than the operations it saves.
__device__ __forceinline__ void sw_split(const Phys& ph, R rho, R u, R v, R w, R c, R k1, R k2, R k3,
                                         R sig, R fp[5], R fm[5], int axis = -1)
{
    const R gm1 = pk<R>(ph.gm1, ph.gm1f);
    const R gm1x2 = gm1 + gm1;
    const R uk = axis == 0 ? u : (axis == 1 ? v : (axis == 2 ? w : mad(k3, w, mad(k2, v, k1 * u))));
    const R V = sig * uk;
    const R cs = c * sig;
    const R l4 = V - cs, l5 = V + cs;
    const R q2 = mad(w, w, mad(v, v, u * u));
    const R H = mad(c * c, pk<R>(ph.inv_gm1, ph.inv_gm1f), (R)0.5 * q2);
    const R a = rho * pk<R>(ph.inv2g, ph.inv2gf);
    const R gq = gm1 * q2;
    const R ac = a * c;
    {
        const R l1 = pos_part(V);
        const R a4 = pos_part(l4);
        const R a5 = pos_part(l5);
        const R s = a4 + a5, dl = a5 - a4;
        const R f0 = a * mad(gm1x2, l1, s);
        const R t = ac * dl;
        fp[0] = f0;
        if (axis >= 0) {
            fp[1] = axis == 0 ? mad(u, f0, t) : u * f0;
            fp[2] = axis == 1 ? mad(v, f0, t) : v * f0;
            fp[3] = axis == 2 ? mad(w, f0, t) : w * f0;
        } else {
            fp[1] = mad(u, f0, t * k1);
            fp[2] = mad(v, f0, t * k2);
            fp[3] = mad(w, f0, t * k3);
        }
        fp[4] = mad(t, uk, a * mad(l1, gq, s * H));
    }
    {
        const R l1 = neg_part(V);
        const R a4 = neg_part(l4);
        const R a5 = neg_part(l5);
        const R s = a4 + a5, dl = a5 - a4;
        const R f0 = a * mad(gm1x2, l1, s);
        const R t = ac * dl;
        fm[0] = f0;
        if (axis >= 0) {
            fm[1] = axis == 0 ? mad(u, f0, t) : u * f0;
            fm[2] = axis == 1 ? mad(v, f0, t) : v * f0;
            fm[3] = axis == 2 ? mad(w, f0, t) : w * f0;
        } else {
            fm[1] = mad(u, f0, t * k1);
            fm[2] = mad(v, f0, t * k2);
            fm[3] = mad(w, f0, t * k3);
        }
        fm[4] = mad(t, uk, a * mad(l1, gq, s * H));
    }
}

// ---------------------------------------------------------------------------
// reconstructions at the face j+1/2 from 7 upwind-ordered values
// v[0..6] = f_{j-3..j+3} (plus side) or f_{j+4..j-2} (minus side, mirrored)
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R ud7(const R v[7])
{
    // Eq. 41
    R r = ((R)(-3.0 / 420.0)) * v[0];
    r = mad((R)(25.0 / 420.0), v[1], r);
    r = mad((R)(-101.0 / 420.0), v[2], r);
    r = mad((R)(319.0 / 420.0), v[3], r);
    r = mad((R)(214.0 / 420.0), v[4], r);
    r = mad((R)(-38.0 / 420.0), v[5], r);
    return mad((R)(4.0 / 420.0), v[6], r);
}

// Smoothness indicator as a weighted sum of squares of constant-annihilating
// linear combinations (derivative coefficients of the sub-stencil polynomial):
// its rounding error scales with |f| sqrt(beta) rather than |f|^2.
template <class R, int NR, int NS>
__device__ __forceinline__ R beta_rows(const double (&S)[NS], const double (&SD)[NR], const R* f)
{
    constexpr int r = NS / NR;
    R b = (R)0;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        R h = (R)S[i * r] * f[0];
#pragma unroll
        for (int l = 1; l < r; ++l) h = mad((R)S[i * r + l], f[l], h);
        b = i == 0 ? (R)SD[0] * (h * h) : mad((R)SD[i], h * h, b);
    }
    return b;
}

template <class R>
__device__ __forceinline__ R dot4(const double (&c)[4], const R* v)
{
    return mad((R)c[3], v[3], mad((R)c[2], v[2], mad((R)c[1], v[1], (R)c[0] * v[0])));
}
template <class R>
__device__ __forceinline__ R dot3(const double (&c)[3], const R* v)
{
    return mad((R)c[2], v[2], mad((R)c[1], v[1], (R)c[0] * v[0]));
}

// WENO7 (Balsara-Shu) on v[0..6]; one division (weights over a common
// denominator, the division hoisting the paper describes).  isc = 1/sigma^2
// of the face: the indicators are measured on the flux per unit face area.
template <class R>
__device__ __forceinline__ R weno7(const R v[7], R eps, R isc)
{
    constexpr double D[4] = W7_D;
    constexpr double SD[3] = W7_SD;
    constexpr double C0[4] = W7_C0, C1[4] = W7_C1, C2[4] = W7_C2, C3[4] = W7_C3;
    constexpr double S0[12] = W7_S0, S1[12] = W7_S1, S2[12] = W7_S2, S3[12] = W7_S3;
    const R q0 = dot4<R>(C0, v + 0), q1 = dot4<R>(C1, v + 1), q2 = dot4<R>(C2, v + 2), q3 = dot4<R>(C3, v + 3);
    R b0 = mad(isc, beta_rows<R>(S0, SD, v + 0), eps);
    R b1 = mad(isc, beta_rows<R>(S1, SD, v + 1), eps);
    R b2 = mad(isc, beta_rows<R>(S2, SD, v + 2), eps);
    R b3 = mad(isc, beta_rows<R>(S3, SD, v + 3), eps);
    R t0 = b0 * b0, t1 = b1 * b1, t2 = b2 * b2, t3 = b3 * b3;
    R w0, w1, w2, w3;
    if (sizeof(R) == 8) {
        R p01 = t0 * t1, p23 = t2 * t3;
        w0 = (R)D[0] * t1 * p23; w1 = (R)D[1] * t0 * p23;
        w2 = (R)D[2] * t3 * p01; w3 = (R)D[3] * t2 * p01;
    } else {
        // FP32: products of three squared indicators (>= eps^6) would reach
        // the denormal range, so divide per candidate
        w0 = (R)D[0] / t0; w1 = (R)D[1] / t1; w2 = (R)D[2] / t2; w3 = (R)D[3] / t3;
    }
    return mad(w3, q3, mad(w2, q2, mad(w1, q1, w0 * q0))) / (((w0 + w1) + w2) + w3);
}

// WENO5 (Jiang-Shu) on v[1..5] = f_{j-2..j+2}; mask bit k drops sub-stencil k
// (the boundary closure of Section 2.2.4).
template <class R>
__device__ __forceinline__ R weno5(const R v[7], R eps, R isc, int mask)
{
    constexpr double D[3] = W5_D;
    constexpr double SD[2] = W5_SD;
    constexpr double C0[3] = W5_C0, C1[3] = W5_C1, C2[3] = W5_C2;
    constexpr double S0[6] = W5_S0, S1[6] = W5_S1, S2[6] = W5_S2;
    const R q0 = dot3<R>(C0, v + 1), q1 = dot3<R>(C1, v + 2), q2 = dot3<R>(C2, v + 3);
    R b0 = mad(isc, beta_rows<R>(S0, SD, v + 1), eps);
    R b1 = mad(isc, beta_rows<R>(S1, SD, v + 2), eps);
    R b2 = mad(isc, beta_rows<R>(S2, SD, v + 3), eps);
    R t0 = b0 * b0, t1 = b1 * b1, t2 = b2 * b2;
    R w0, w1, w2;
    if (sizeof(R) == 8) {
        w0 = (R)D[0] * t1 * t2; w1 = (R)D[1] * t0 * t2; w2 = (R)D[2] * t0 * t1;
    } else {
        w0 = (R)D[0] / t0; w1 = (R)D[1] / t1; w2 = (R)D[2] / t2;
    }
    if (mask & 1) w0 = (R)0;
    if (mask & 2) w1 = (R)0;
    if (mask & 4) w2 = (R)0;
    return mad(w2, q2, mad(w1, q1, w0 * q0)) / ((w0 + w1) + w2);
}

// one face value from upwind-ordered values; use: 0 UD7, 1 WENO7, 2 WENO5
template <class R>
__device__ __forceinline__ R recon(int use, const R v[7], R eps, R isc, int mask)
{
    if (use == 0) return ud7<R>(v);
    if (use == 1) return weno7<R>(v, eps, isc);
    return weno5<R>(v, eps, isc, mask);
}

// 1/sigma_{j+1/2}^2 with sigma_{j+1/2} = (sigma_j + sigma_{j+1})/2, sigma =
// |grad d|/J the face-area scale of the nodes' split fluxes (reading R23)
template <class R>
__device__ __forceinline__ R face_iscale(R sa, R sb)
{
    const R s = sa + sb;
    return (R)4 / (s * s);
}

// Face flux at j+1/2 of component q from the 8 node values f_{j-3..j+4}.
template <class R>
__device__ __forceinline__ R face_flux(int use, const R fp8[8], const R fm8[8], R eps, R isc, int maskp,
                                       int maskm)
{
    R vp[7], vm[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        vp[o] = fp8[o];
        vm[o] = fm8[7 - o];
    }
    return recon<R>(use, vp, eps, isc, maskp) + recon<R>(use, vm, eps, isc, maskm);
}

// ---------------------------------------------------------------------------
// characteristic-variable reconstruction of one WENO face (Sec. 2.2.2,
// Eq. 31-40): the interface state U_{j+1/2} = (U_j + U_{j+1})/2 (Eq. 32,
// from the FP64 state), the unit normal n of the face, the left eigenvectors
// S (Eq. 35) applied to the split fluxes of the eight stencil nodes, one
// reconstruction per characteristic field, and the right eigenvectors
// (Eq. 34) applied to the result.  fpl(o, q) / fml(o, q): component q of
// f+ / f- at stencil node j-3+o, o = 0..7.
// ---------------------------------------------------------------------------
template <class R, class FP, class FM>
__device__ __forceinline__ void face_flux_char(const Phys& ph, int use, R eps, R isc, int mp, int mm,
                                               const double* __restrict__ U, long long N, long long na,
                                               long long nb, R n1, R n2, R n3, FP fpl, FM fml, R out[5])
{
    const double r0 = 0.5 * (U[na] + U[nb]);
    const double r1 = 0.5 * (U[N + na] + U[N + nb]);
    const double r2 = 0.5 * (U[2 * N + na] + U[2 * N + nb]);
    const double r3 = 0.5 * (U[3 * N + na] + U[3 * N + nb]);
    const double r4 = 0.5 * (U[4 * N + na] + U[4 * N + nb]);
    const R rho = (R)r0, ri = (R)1 / rho;
    const R u = (R)r1 * ri, v = (R)r2 * ri, w = (R)r3 * ri;
    const R V = (R)0.5 * (u * u + v * v + w * w);                         // Eq. 25
    const R p = pk<R>(ph.gm1, ph.gm1f) * ((R)r4 - rho * V);
    const R c2 = pk<R>(ph.gamma, ph.gammaf) * p * ri;
    const R c = sqrt(c2);
    const R H = V + c2 * pk<R>(ph.inv_gm1, ph.inv_gm1f);                  // Eq. 36
    const R kap = pk<R>(ph.gm1, ph.gm1f) / c2, kap1 = (R)0.5 * kap;       // Eq. 37
    const R chi = (R)0.5 / c;
    R l1, l2, l3;                                                          // Eq. 39
    if (fabs(n3) <= fabs(n2)) {
        const R r = (R)1 / sqrt(n1 * n1 + n2 * n2);
        l1 = -n2 * r; l2 = n1 * r; l3 = (R)0;
    } else {
        const R r = (R)1 / sqrt(n1 * n1 + n3 * n3);
        l1 = -n3 * r; l2 = (R)0; l3 = n1 * r;
    }
    const R m1 = n2 * l3 - n3 * l2, m2 = n3 * l1 - n1 * l3, m3 = n1 * l2 - n2 * l1;  // Eq. 40
    const R un = u * n1 + v * n2 + w * n3, ul = u * l1 + v * l2 + w * l3, um = u * m1 + v * m2 + w * m3;
    R gh[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        R s0, s1, s2, s3, s4;  // row k of S (Eq. 35)
        if (k == 0) { s0 = (R)1 - kap * V; s1 = kap * u; s2 = kap * v; s3 = kap * w; s4 = -kap; }
        else if (k == 1) { s0 = -ul; s1 = l1; s2 = l2; s3 = l3; s4 = (R)0; }
        else if (k == 2) { s0 = -um; s1 = m1; s2 = m2; s3 = m3; s4 = (R)0; }
        else if (k == 3) {
            s0 = kap1 * V + chi * un; s1 = -chi * n1 - kap1 * u; s2 = -chi * n2 - kap1 * v;
            s3 = -chi * n3 - kap1 * w; s4 = kap1;
        } else {
            s0 = kap1 * V - chi * un; s1 = chi * n1 - kap1 * u; s2 = chi * n2 - kap1 * v;
            s3 = chi * n3 - kap1 * w; s4 = kap1;
        }
        R vp[7], vm[7];
#pragma unroll
        for (int o = 0; o < 7; ++o) {
            vp[o] = s0 * fpl(o, 0) + s1 * fpl(o, 1) + s2 * fpl(o, 2) + s3 * fpl(o, 3) + s4 * fpl(o, 4);
            vm[o] = s0 * fml(7 - o, 0) + s1 * fml(7 - o, 1) + s2 * fml(7 - o, 2) + s3 * fml(7 - o, 3) +
                    s4 * fml(7 - o, 4);
        }
        gh[k] = recon<R>(use, vp, eps, isc, mp) + recon<R>(use, vm, eps, isc, mm);
    }
    // columns of S^-1 (Eq. 34)
    out[0] = gh[0] + gh[3] + gh[4];
    out[1] = u * gh[0] + l1 * gh[1] + m1 * gh[2] + (u - c * n1) * gh[3] + (u + c * n1) * gh[4];
    out[2] = v * gh[0] + l2 * gh[1] + m2 * gh[2] + (v - c * n2) * gh[3] + (v + c * n2) * gh[4];
    out[3] = w * gh[0] + l3 * gh[1] + m3 * gh[2] + (w - c * n3) * gh[3] + (w + c * n3) * gh[4];
    out[4] = V * gh[0] + ul * gh[1] + um * gh[2] + (H - c * un) * gh[3] + (H + c * un) * gh[4];
}

// unit normal of face j+1/2 in direction d from the metric vectors alpha of
// its two nodes (metric indices ma, mb)
template <class R>
__device__ __forceinline__ void face_normal(const Geo& g, int d, long long ma, long long mb, R* n1, R* n2, R* n3)
{
    const R a1 = metr<R>(g, M_ALPHA + 3 * d, ma) + metr<R>(g, M_ALPHA + 3 * d, mb);
    const R a2 = metr<R>(g, M_ALPHA + 3 * d + 1, ma) + metr<R>(g, M_ALPHA + 3 * d + 1, mb);
    const R a3 = metr<R>(g, M_ALPHA + 3 * d + 2, ma) + metr<R>(g, M_ALPHA + 3 * d + 2, mb);
    const R r = (R)1 / sqrt(a1 * a1 + a2 * a2 + a3 * a3);
    *n1 = a1 * r;
    *n2 = a2 * r;
    *n3 = a3 * r;
}

// scheme class of face j+1/2 (nodes j-3..j+4 of one line): returns use and masks.
// Non-periodic lines: a face whose stencil leaves [0, n-1] uses masked WENO5.
__device__ __forceinline__ int face_use(const Phys& ph, int per, int n, int j, int cmax, int* maskp,
                                        int* maskm)
{
    *maskp = 0;
    *maskm = 0;
    if (!per && (j - 3 < 0 || j + 4 > n - 1)) {
        int mp = 0, mm = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // plus side: nodes j-2+k .. j+k ; minus side: nodes j+1-k .. j+3-k
            if (j - 2 + k < 0 || j + k > n - 1) mp |= 1 << k;
            if (j + 1 - k < 0 || j + 3 - k > n - 1) mm |= 1 << k;
        }
        *maskp = mp;
        *maskm = mm;
        return 2;
    }
    switch (ph.scheme) {
    case 0: return 0;
    case 1: return 2;
    case 2: return 1;
    default: return cmax;
    }
}

// ---------------------------------------------------------------------------
// central first derivative in index space with the closures of Section 2.3
// ---------------------------------------------------------------------------
// central first-derivative stencils from the differences d_k = f(m+k) - f(m-k)
template <class R>
__device__ __forceinline__ R cen8(R d1, R d2, R d3, R d4)
{
    return mad((R)(-3.0 / 840.0), d4, mad((R)(32.0 / 840.0), d3, mad((R)(-168.0 / 840.0), d2, (R)(672.0 / 840.0) * d1)));
}
template <class R>
__device__ __forceinline__ R cen6(R d1, R d2, R d3)
{
    return mad((R)(1.0 / 60.0), d3, mad((R)(-9.0 / 60.0), d2, (R)(45.0 / 60.0) * d1));
}

template <class R, class Ld>
__device__ __forceinline__ R dcentral(int order, int per, int n, int m, Ld f)
{
    if (per) {
        auto d = [&](int k) { return f(wrapi(m + k, n)) - f(wrapi(m - k, n)); };
        if (order == 8) return cen8<R>(d(1), d(2), d(3), d(4));
        return cen6<R>(d(1), d(2), d(3));
    }
    if (m == 0) return mad((R)(-0.5), f(2), mad((R)2, f(1), (R)(-1.5) * f(0)));
    if (m == n - 1) return mad((R)0.5, f(n - 3), mad((R)(-2), f(n - 2), (R)1.5 * f(n - 1)));
    auto d = [&](int k) { return f(m + k) - f(m - k); };
    if (m == 1 || m == n - 2) return (R)0.5 * d(1);
    if (m == 2 || m == n - 3) return mad((R)(-1.0 / 12.0), d(2), (R)(8.0 / 12.0) * d(1));
    if (m == 3 || m == n - 4 || order == 6) return cen6<R>(d(1), d(2), d(3));
    return cen8<R>(d(1), d(2), d(3), d(4));
}

// whether direction d of the viscous derivatives is folded: FP64 only (the
// FP64 pipe is what bounds that form; in FP32 the extra branches cost more
// than the multiply they save)
template <class R>
__device__ __forceinline__ bool fold_dir(const Geo& g, int d)
{
    return sizeof(R) == 8 && g.gfold[d];
}

// Cartesian derivative along a folded direction d (Geo::gfold): the central
// stencil of the viscous order with coefficients c_k d_x (one multiply per
// derivative fewer than differentiating and then applying the metric)
template <class R, class Ld>
__device__ __forceinline__ R dcentral_folded(const Geo& g, int order, int d, int m, Ld f)
{
    R c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = (R)g.gsc[d][k];
    auto dd = [&](int k) { return f(m + k) - f(m - k); };
    if (order == 8) return mad(c[3], dd(4), mad(c[2], dd(3), mad(c[1], dd(2), c[0] * dd(1))));
    return mad(c[2], dd(3), mad(c[1], dd(2), c[0] * dd(1)));
}

// central derivative on a tile: f(m) takes unwrapped line positions, so the
// periodic form needs no wrap (the tile rows already hold the wrapped nodes)
template <class R, class Ld>
__device__ __forceinline__ R dcentral_tile(int order, int per, int n, int m, Ld f)
{
    if (per) {
        auto d = [&](int k) { return f(m + k) - f(m - k); };
        if (order == 8) return cen8<R>(d(1), d(2), d(3), d(4));
        return cen6<R>(d(1), d(2), d(3));
    }
    return dcentral<R>(order, 0, n, m, f);
}

// the central derivative of the viscous divergence in the sweeps; P8: the
// swept line is periodic and the order 8, known at compile time (the same
// operations without the order and closure decisions)
template <class R, bool P8, class Ld>
__device__ __forceinline__ R dvisc(int order, int per, int n, int m, Ld f)
{
    if constexpr (P8) {
        auto d = [&](int k) { return f(m + k) - f(m - k); };
        return cen8<R>(d(1), d(2), d(3), d(4));
    } else {
        return dcentral_tile<R>(order, per, n, m, f);
    }
}

// ---------------------------------------------------------------------------
// viscous fluxes at nodes (Eqs. 9-15 with readings R13-R15)
// ---------------------------------------------------------------------------
// Power law mu = T^omega, table-driven (a table method in the manner of
// Tang, ACM TOMS 15, 1989).  With T = 2^e m, m in [1, 2), m_k = 1 + k/256 the
// node below m (k = the top 8 fraction bits) and delta = (m - m_k)/m_k in
// [0, 1/256):
//     T^omega = 2^(e omega) m_k^omega (1 + delta)^omega,
// the last factor by its binomial series to delta^6 (FP64; the next term is
// below 2^-56) or delta^3 (FP32).  The exponent and k come from the bit
// pattern (integer pipe); 2^(e omega) for e in [-64, 63], m_k^omega and 1/m_k
// are tables built per context on the host; the FP64 form takes 10 FP64
// operations where exp(omega log T) takes about 45.  Relative error a few
// units of rounding (the two table entries, the series and three roundings).
// Temperatures outside [2^-64, 2^64), non-positive or not finite, and
// contexts without tables, take exp(omega log T).
enum { PT_M = 0, PT_INV = 256, PT_E = 512, PT_COUNT = 640 };

__device__ __forceinline__ double power_law(const Phys& ph, double T)
{
    const long long b = __double_as_longlong(T);
    const int e = (int)(b >> 52) - 1023;
    if (ph.powtab && (unsigned)(e + 64) < 128u) {
        const double* t = ph.powtab;
        const int k = (int)((b >> 44) & 0xff);
        const double m = __longlong_as_double((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
        const double mk = __longlong_as_double(0x3ff0000000000000ll | ((long long)k << 44));
        const double d = (m - mk) * __ldg(t + PT_INV + k);
        double p = ph.pc[5];
#pragma unroll
        for (int j = 4; j >= 0; --j) p = mad(p, d, ph.pc[j]);
        p = mad(p, d, 1.0);
        return (p * __ldg(t + PT_M + k)) * __ldg(t + PT_E + e + 64);
    }
    return exp(ph.omega * log(T));
}

__device__ __forceinline__ float power_law(const Phys& ph, float T)
{
    const int b = __float_as_int(T);
    const int e = (b >> 23) - 127;
    if (ph.powtabf && (unsigned)(e + 64) < 128u) {
        const float* t = ph.powtabf;
        const int k = (b >> 15) & 0xff;
        const float m = __int_as_float((b & 0x007fffff) | 0x3f800000);
        const float mk = __int_as_float(0x3f800000 | (k << 15));
        const float d = (m - mk) * __ldg(t + PT_INV + k);
        float p = mad(mad(ph.pcf[2], d, ph.pcf[1]), d, ph.pcf[0]);
        p = mad(p, d, 1.0f);
        return (p * __ldg(t + PT_M + k)) * __ldg(t + PT_E + e + 64);
    }
    return powf(T, ph.omegaf);
}

__device__ __forceinline__ double viscosity(const Phys& ph, double T)
{
    if (ph.visc_law == 1) return power_law(ph, T);
    double s = ph.suth_s;
    return T * sqrt(T) * (1.0 + s) / (T + s);
}

__device__ __forceinline__ float viscosity(const Phys& ph, float T)
{
    if (ph.visc_law == 1) return power_law(ph, T);
    float s = ph.suth_sf;
    return T * sqrtf(T) * (1.0f + s) / (T + s);
}

// mu(T) of n temperatures through the kernels' routine (a check of it)
template <class R>
__global__ void k_eval_viscosity(Phys ph, const double* T, double* mu, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) mu[t] = (double)viscosity(ph, (R)T[t]);
}

// Cartesian gradients q_x = xi_x q_xi + eta_x q_eta + zeta_x q_zeta, ... of
// u, v, w, T (Eq. 9-14 through the metrics of Eq. 3).  On a box whose metric
// matrices are diagonal the zero terms of the sums are skipped: a fused
// multiply-add with a zero factor adds exactly nothing, so both forms give
// the same bits.
template <class R>
__device__ __forceinline__ void cartesian_gradients(const Geo& g, long long mi, const R dq[4][3], R gr[4][3])
{
    if (g.diag) {
        // folded directions arrive as Cartesian derivatives already
        const R m0 = metr<R>(g, M_RAW + 0, mi), m1 = metr<R>(g, M_RAW + 4, mi), m2 = metr<R>(g, M_RAW + 8, mi);
#pragma unroll
        for (int var = 0; var < 4; ++var) {
            gr[var][0] = fold_dir<R>(g, 0) ? dq[var][0] : m0 * dq[var][0];
            gr[var][1] = fold_dir<R>(g, 1) ? dq[var][1] : m1 * dq[var][1];
            gr[var][2] = fold_dir<R>(g, 2) ? dq[var][2] : m2 * dq[var][2];
        }
        return;
    }
    R mraw[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) mraw[e] = metr<R>(g, M_RAW + e, mi);
#pragma unroll
    for (int var = 0; var < 4; ++var)
#pragma unroll
        for (int x = 0; x < 3; ++x)
            gr[var][x] = mad(mraw[6 + x], dq[var][2], mad(mraw[3 + x], dq[var][1], mraw[x] * dq[var][0]));
}

// viscous fluxes at a node: Fv_d = alpha_d . (tau, Theta) with alpha_d =
// grad(d)/J (Eq. 9-11); diagonal metrics keep the one nonzero term
template <class R>
__device__ __forceinline__ void store_visc_fluxes(const Geo& g, long long mi, long long n, const R tau[3][3],
                                                  const R Th[3], R* __restrict__ Fv)
{
    const long long N = g.N;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (g.diag) {
            const R ad = metr<R>(g, M_ALPHA + 4 * d, mi);
#pragma unroll
            for (int row = 0; row < 3; ++row) Fv[(long long)(4 * d + row) * N + n] = ad * tau[d][row];
            Fv[(long long)(4 * d + 3) * N + n] = ad * Th[d];
            continue;
        }
        R a0 = metr<R>(g, M_ALPHA + 3 * d, mi), a1 = metr<R>(g, M_ALPHA + 3 * d + 1, mi),
          a2 = metr<R>(g, M_ALPHA + 3 * d + 2, mi);
#pragma unroll
        for (int row = 0; row < 3; ++row)
            Fv[(long long)(4 * d + row) * N + n] = mad(a2, tau[2][row], mad(a1, tau[1][row], a0 * tau[0][row]));
        Fv[(long long)(4 * d + 3) * N + n] = mad(a2, Th[2], mad(a1, Th[1], a0 * Th[0]));
    }
}

// fluxes of one node from its derivatives of u, v, w, T in index space
// (gradients through the metrics, mu(T), tau and Theta of Eq. 12-15)
template <class R>
__device__ __forceinline__ void visc_node_flux(const Geo& g, const Phys& ph, long long n, int i, int j, const R dq[4][3],
                                               R T, R u, R v, R w, R* __restrict__ Fv)
{
    const long long mi = midx(g, i, j, n);
    R gr[4][3];
    cartesian_gradients<R>(g, mi, dq, gr);
    const R mu = viscosity(ph, T);
    const R mr = mu * pk<R>(ph.invRe, ph.invRef);
    const R div = (gr[0][0] + gr[1][1]) + gr[2][2];
    R tau[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            tau[a][b] = a == b ? mr * mad((R)(-2.0 / 3.0), div, gr[a][a] + gr[a][a]) : mr * (gr[a][b] + gr[b][a]);
    const R kc = mu * pk<R>(ph.kcoef, ph.kcoeff);
    R Th[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Th[a] = mad(kc, gr[3][a], mad(w, tau[a][2], mad(v, tau[a][1], u * tau[a][0])));
    store_visc_fluxes<R>(g, mi, n, tau, Th, Fv);
}

// YB > 0: CTAs of 32 x YB nodes in an x-y tile (the y neighbours of a tile's
// nodes are shared through L1); YB = 0: CTAs along one x row.
// P8: every direction periodic and the viscous order 8 (known at compile
// time: the derivatives take the interior stencil with no order or closure
// decisions; the same operations as the general path)
// SENS (FP32 only): the node's plain shock-sensor class (Eq. 42-43, the
// operations of sensor32_body in the same order) is formed here too, from the
// pressures at m-1 and m+1 of the stencil offsets the derivatives use; the
// stage then needs no separate sensor launch
template <class R, int YB = 0, bool P8 = false, bool SENS = false>
__device__ __forceinline__ void visc_node_body(const SweepArgs& A, uint3 vb)
{
    const Geo& g = A.g;
    const Phys& ph = A.ph;
    const R* __restrict__ P = (const R*)A.P;
    R* __restrict__ Fv = (R*)A.Fv;
    const long long N = g.N;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int ord = ph.vorder;
    int i, j, k;
    long long n;
    if constexpr (YB > 0) {
        i = vb.x * 32 + threadIdx.x;
        j = vb.y * YB + threadIdx.y;
        k = vb.z;
    } else {
        i = vb.x * blockDim.x + threadIdx.x;
        j = vb.y;
        k = vb.z;
    }
    n = (long long)i + (long long)g.nx * ((long long)j + (long long)g.ny * k);
    if (i < g.nx && j < g.ny)
    {
        const int st[3] = {1, nx, nx * ny};
        const int pos[3] = {i, j, k};
        const int nd[3] = {nx, ny, nz};
        // element offsets of the line positions m-4..m+4 in each direction,
        // computed once and shared by the four fields (periodic lines wrap)
        int off[3][9];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // only nodes within 4 of the ends of a periodic line need wrapping
            const bool wrap = g.per[d] && (pos[d] < 4 || pos[d] + 4 >= nd[d]);
#pragma unroll
            for (int t = 0; t < 9; ++t)
                off[d][t] = wrap ? (wrapi(pos[d] + t - 4, nd[d]) - pos[d]) * st[d] : (t - 4) * st[d];
        }
#ifdef CFD_BOUNDS_CHECK
        {
            bool inb = true;
            // positions a derivative reads: all 9 on periodic lines, those
            // inside the line otherwise (the boundary closures stay inside)
            for (int d = 0; d < 3; ++d)
                for (int t = 0; t < 9; ++t) {
                    const int q = pos[d] + t - 4;
                    if (g.per[d] || (q >= 0 && q < nd[d])) inb = inb && in_range(A.err, n + off[d][t], N);
                }
            if (!inb) return;
        }
#endif
        // the plane that the CTAs one stencil reach further in zeta will
        // read first (k + 5) requested into L2 now
        if constexpr (YB > 0) {
            const int kp = k + 5;
            if (g.per[2] || kp < nz) {
                const long long np = n + (long long)((g.per[2] ? wrapi(kp, nz) : kp) - k) * st[2];
                if (in_range(A.err, np, N)) {
#pragma unroll
                    for (int var = 0; var < 4; ++var) prefetch_l2(P + (long long)(var < 3 ? var + 1 : 5) * N + np);
                    if constexpr (SENS) prefetch_l2(P + 4 * N + np);
                }
            }
        }
        // dq[var][d]: var = u, v, w, T (P rows 1, 2, 3, 5)
        R dq[4][3];
#pragma unroll
        for (int var = 0; var < 4; ++var) {
            const R* f = P + (long long)(var < 3 ? var + 1 : 5) * N + n;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int m = pos[d];
                auto ld = [&](int mm) { return __ldg(f + off[d][mm - m + 4]); };
                if constexpr (P8) {
                    auto dd = [&](int kk) { return ld(m + kk) - ld(m - kk); };
                    dq[var][d] = fold_dir<R>(g, d) ? dcentral_folded<R>(g, 8, d, m, ld)
                                                   : cen8<R>(dd(1), dd(2), dd(3), dd(4));
                } else {
                    dq[var][d] = fold_dir<R>(g, d) ? dcentral_folded<R>(g, ord, d, m, ld)
                                                   : dcentral_tile<R>(ord, g.per[d], nd[d], m, ld);
                }
            }
        }
        visc_node_flux<R>(g, ph, n, i, j, dq, P[5 * N + n], P[N + n], P[2 * N + n], P[3 * N + n], Fv);
        if constexpr (SENS) {
            static_assert(sizeof(R) == sizeof(float), "the fused sensor is the FP32 one");
            const float* __restrict__ p = (const float*)P + 4 * N + n;
            const float p0 = p[0];
            float th = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int m = pos[d];
                if (!P8 && !g.per[d] && (m == 0 || m == nd[d] - 1)) continue;  // reading R4
                const float pm = p[off[d][3]];
                const float pp = p[off[d][5]];
                const float p2 = p0 + p0;
                th += fabsf((p2 - pm) - pp) / ((pm + p2) + pp);
            }
            A.cls_io[n] = th <= ph.th1f ? 0 : (th <= ph.th2f ? 1 : 2);
        }
    }
}

// Viscous node fluxes, 2.5-D form: a CTA owns 32 x 8 nodes of an (x, y) tile
// and walks along zeta over a segment of TZ planes.  Each plane of u, v, w, T
// with a 4-node x/y halo is staged once in a 9-plane shared ring; the x and y
// derivatives of the centre plane and the zeta derivatives all come from
// shared memory, so every value is read from L2/HBM about 2.5 times instead of
// once per stencil use.  Same operations, in the same order, as k_visc_flux.
template <class R>
constexpr size_t visc25_smem_bytes()
{
    return (size_t)9 * 4 * 16 * 40 * sizeof(R);
}

template <class R, int TZ>
__device__ __forceinline__ void visc25_body(const SweepArgs& A, uint3 vb)
{
    const Geo& g = A.g;
    const Phys& ph = A.ph;
    const R* __restrict__ P = (const R*)A.P;
    R* __restrict__ Fv = (R*)A.Fv;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* ring = reinterpret_cast<R*>(smem_raw);  // [9][4][16][40]
    constexpr int PL = 4 * 16 * 40;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long N = g.N;
    const int x0 = vb.x * 32, y0 = vb.y * 8;
    const int zlo = vb.z * TZ, zhi = min(zlo + TZ, nz);
    const int i = x0 + tx, j = y0 + ty;
    const bool own = i < nx && j < ny;
    const int ord = ph.vorder;
    const R* fld[4] = {P + N, P + 2 * N, P + 3 * N, P + 5 * N};
    for (int z = zlo - 4; z < zhi + 4; ++z) {
        // stage plane z (with its x/y halo) into ring slot z mod 9
        const int slot = ((z % 9) + 9) % 9;
        R* pl = ring + (size_t)slot * PL;
        const bool zin = g.per[2] || (z >= 0 && z < nz);
        const int zz = g.per[2] ? wrapi(z, nz) : z;
        for (int t = threadIdx.x; t < 16 * 40; t += 256) {
            const int hy = t / 40, hx = t - hy * 40;
            int gx = x0 - 4 + hx, gy = y0 - 4 + hy;
            bool ok = zin;
            if (g.per[0]) gx = wrapi(gx, nx);
            else ok = ok && gx >= 0 && gx < nx;
            if (g.per[1]) gy = wrapi(gy, ny);
            else ok = ok && gy >= 0 && gy < ny;
            const long long nn = ok ? (long long)gx + (long long)nx * ((long long)gy + (long long)ny * zz) : 0;
#pragma unroll
            for (int f = 0; f < 4; ++f) pl[f * 640 + t] = ok ? __ldg(fld[f] + nn) : (R)0;
        }
        __syncthreads();
        const int zc = z - 4;  // output plane: its +-4 neighbours are all staged now
        if (zc >= zlo && own) {
            const R* c = ring + (size_t)(((zc % 9) + 9) % 9) * PL;
            const int hx = tx + 4, hy = ty + 4;
            R dq[4][3];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const R* cf = c + f * 640;
                auto lx = [&](int mm) { return cf[hy * 40 + hx + (mm - i)]; };
                auto ly = [&](int mm) { return cf[(hy + (mm - j)) * 40 + hx]; };
                auto lz = [&](int mm) { return ring[(size_t)(((mm % 9) + 9) % 9) * PL + f * 640 + hy * 40 + hx]; };
                dq[f][0] = fold_dir<R>(g, 0) ? dcentral_folded<R>(g, ord, 0, i, lx)
                                             : dcentral_tile<R>(ord, g.per[0], nx, i, lx);
                dq[f][1] = fold_dir<R>(g, 1) ? dcentral_folded<R>(g, ord, 1, j, ly)
                                             : dcentral_tile<R>(ord, g.per[1], ny, j, ly);
                dq[f][2] = fold_dir<R>(g, 2) ? dcentral_folded<R>(g, ord, 2, zc, lz)
                                             : dcentral_tile<R>(ord, g.per[2], nz, zc, lz);
            }
            const long long n = (long long)i + (long long)nx * ((long long)j + (long long)ny * zc);
            const R* cu = c;
            visc_node_flux<R>(g, ph, n, i, j, dq, P[5 * N + n], cu[hy * 40 + hx], cu[640 + hy * 40 + hx],
                              cu[1280 + hy * 40 + hx], Fv);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// the directional sweeps
// ---------------------------------------------------------------------------
// epilogue modes
enum { EP_STORE = 0, EP_ACCUM = 1, EP_FINAL_RHS = 2, EP_FINAL_RK = 3 };


// the epilogue's operands of node nn (the accumulator; U and U^n for the RK
// update) requested into L2 ahead of the epilogue
template <class R, int EP>
__device__ __forceinline__ void prefetch_epilogue(const SweepArgs& A, long long nn)
{
    if (EP == EP_STORE) return;
    const long long N = A.g.N;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        prefetch_l2((const R*)A.R + q * N + nn);
        if (EP == EP_FINAL_RK) {
            prefetch_l2(A.U + q * N + nn);
            if (A.rk_a != 0.0) prefetch_l2(A.Un + q * N + nn);
        }
    }
}

// the inputs a sweep along direction d reads at node nn (rho, u, v, w, c,
// the class, the viscous fluxes of d) requested into L2
template <class R>
__device__ __forceinline__ void prefetch_row_inputs(const SweepArgs& A, int d, long long nn)
{
    const long long N = A.g.N;
    const R* P = (const R*)A.P;
#pragma unroll
    for (int f = 0; f < 4; ++f) prefetch_l2(P + f * N + nn);
    prefetch_l2(P + 6 * N + nn);
    if (A.cls) prefetch_l2(A.cls + nn);
    if (A.Fv) {
#pragma unroll
        for (int c = 0; c < 4; ++c) prefetch_l2((const R*)A.Fv + (long long)(4 * d + c) * N + nn);
    }
}

// RK3 update of one conserved variable, U_out = a U^n + b (U + dt J s), with s
// the summed sweep residual (exact in FP64) and dtJ = dt J formed once per
// node; the first stage (a = 0, b = 1) is a single FMA
__device__ __forceinline__ double rk_combine(const SweepArgs& A, double dtJ, double s, double u, double un)
{
    const double y = mad(dtJ, s, u);
    return A.rk_a == 0.0 && A.rk_b == 1.0 ? y : mad(A.rk_a, un, A.rk_b * y);
}

template <class R, int EP>
__device__ __forceinline__ void epilogue(const SweepArgs& A, long long n, int i, int j, int k, const R val[5])
{
    const long long N = A.g.N;
    if (!in_range(A.err, n, N)) return;
    R* Racc = (R*)A.R;
    if (EP == EP_STORE) {
#pragma unroll
        for (int q = 0; q < 5; ++q) Racc[q * N + n] = val[q];
    } else if (EP == EP_ACCUM) {
#pragma unroll
        for (int q = 0; q < 5; ++q) Racc[q * N + n] += val[q];
    } else {
        const bool bnd = is_bnd(A.g, i, j, k);
        const double J = metv(A.g, M_J, midx(A.g, i, j, n));
        if (EP == EP_FINAL_RHS) {
#pragma unroll
            for (int q = 0; q < 5; ++q) A.Lout[q * N + n] = bnd ? 0.0 : J * to_f64(Racc[q * N + n] + val[q]);
        } else {
            if (bnd) return;  // boundary nodes are set by the boundary conditions
            const double dtJ = *A.dt * J;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const double un = A.rk_a != 0.0 ? A.Un[q * N + n] : 0.0;
                A.Uout[q * N + n] = rk_combine(A, dtJ, to_f64(Racc[q * N + n] + val[q]), A.U[q * N + n], un);
            }
        }
    }
}

// viscous contribution D_d Fv_d at node position m of a line (4 rows -> val[1..4])
template <class R>
__device__ __forceinline__ void visc_div(const SweepArgs& A, int d, long long base, long long stride, int n, int m,
                                         R val[5])
{
    const R* Fv = (const R*)A.Fv;
    const long long N = A.g.N;
#pragma unroll
    for (int row = 0; row < 4; ++row) {
        const R* f = Fv + (long long)(4 * d + row) * N + base;
        val[row + 1] += dcentral<R>(A.ph.vorder, A.g.per[d], n, m,
                                    [&](int mm) { return __ldg(f + (long long)mm * stride); });
    }
}

// primitives a split needs (rho, u, v, w, c), loaded through the read-only path
template <class R>
struct NodePrim {
    R rho, u, v, w, c;
};

template <class R>
__device__ __forceinline__ NodePrim<R> load_prim(const SweepArgs& A, long long n)
{
    const R* __restrict__ P = (const R*)A.P;
    const long long N = A.g.N;
    return {__ldg(P + n), __ldg(P + N + n), __ldg(P + 2 * N + n), __ldg(P + 3 * N + n), __ldg(P + 6 * N + n)};
}

// split fluxes from loaded primitives along direction d; returns sigma
template <class R>
__device__ __forceinline__ R split_prim(const SweepArgs& A, int d, const NodePrim<R>& q, long long mi, R fp[5], R fm[5])
{
    R k1 = metr<R>(A.g, M_K + 3 * d, mi), k2 = metr<R>(A.g, M_K + 3 * d + 1, mi),
      k3 = metr<R>(A.g, M_K + 3 * d + 2, mi), sg = metr<R>(A.g, M_SIG + d, mi);
    if (sizeof(R) == 8 && A.g.diag) sw_split<R>(A.ph, q.rho, q.u, q.v, q.w, q.c, k1, k2, k3, sg, fp, fm, d);
    else sw_split<R>(A.ph, q.rho, q.u, q.v, q.w, q.c, k1, k2, k3, sg, fp, fm);
    return sg;
}

// split fluxes of node (i, j, k) along direction d; returns the node's sigma
template <class R>
__device__ __forceinline__ R node_split(const SweepArgs& A, int d, long long n, int i, int j, R fp[5], R fm[5])
{
    const R* P = (const R*)A.P;
    const long long N = A.g.N;
    const long long mi = midx(A.g, i, j, n);
    R rho = P[n], u = P[N + n], v = P[2 * N + n], w = P[3 * N + n], c = P[6 * N + n];
    R k1 = metr<R>(A.g, M_K + 3 * d, mi), k2 = metr<R>(A.g, M_K + 3 * d + 1, mi),
      k3 = metr<R>(A.g, M_K + 3 * d + 2, mi), sg = metr<R>(A.g, M_SIG + d, mi);
    if (sizeof(R) == 8 && A.g.diag) sw_split<R>(A.ph, rho, u, v, w, c, k1, k2, k3, sg, fp, fm, d);
    else sw_split<R>(A.ph, rho, u, v, w, c, k1, k2, k3, sg, fp, fm);
    return sg;
}

// xi sweep: one CTA per segment of BX nodes of one x-line, halo of 4 nodes.
// CHAR: WENO faces reconstruct characteristic fields (Sec. 2.2.2).
template <class R, int BX, int EP, bool CHAR = false, bool P8 = false>
__device__ __forceinline__ void sweep_x_body(const SweepArgs& A, uint3 vb)
{
    __shared__ __align__(16) R sf[10][BX + 12];  // rows padded so a 12-value window never leaves a row
    __shared__ R sh[5][BX + 1];
    __shared__ R sv[4][BX + 8];
    __shared__ uint8_t sc[BX + 12];
    __shared__ R ss[BX + 12];                    // sigma of the stencil nodes
    __shared__ uint8_t suse[BX + 1];             // per face: use | mask+ << 2 | mask- << 5 (0xff: none)
    __shared__ R sisc[BX + 1];                   // per face: 1/sigma^2 (WENO faces)
    const Geo& g = A.g;
    const int n = g.nx;
    const int per = g.per[0];
    const int j = vb.y, k = vb.z;
    const int lo = per ? 0 : 1;                 // first node that gets a right-hand side
    const int i0 = lo + vb.x * BX;
    const long long row = (long long)n * (j + (long long)g.ny * k);
    const int t = threadIdx.x;
    for (int s = t; s < BX + 8; s += BX) {
        int i = i0 - 4 + s;
        bool ok = per || (i >= 0 && i < n);
        R fp[5], fm[5], sg = (R)0;
        uint8_t c = 0;
        if (ok) ok = in_range(A.err, row + (per ? wrapi(i, n) : i), g.N);
        if (ok) {
            int ii = per ? wrapi(i, n) : i;
            sg = node_split<R>(A, 0, row + ii, ii, j, fp, fm);
            if (A.cls) c = A.cls[row + ii];
            if (A.Fv) {
#pragma unroll
                for (int r = 0; r < 4; ++r) sv[r][s] = ((const R*)A.Fv)[(long long)r * g.N + row + ii];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 5; ++q) fp[q] = fm[q] = (R)0;
            if (A.Fv) {
#pragma unroll
                for (int r = 0; r < 4; ++r) sv[r][s] = (R)0;
            }
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            sf[q][s] = fp[q];
            sf[5 + q][s] = fm[q];
        }
        sc[s] = c;
        ss[s] = sg;
    }
    if (t < 4) {
#pragma unroll
        for (int q = 0; q < 10; ++q) sf[q][BX + 8 + t] = (R)0;
        sc[BX + 8 + t] = 0;
        ss[BX + 8 + t] = (R)0;
    }
    __syncthreads();
    // faces: slot f <-> face (i0-1+f)+1/2 (stencil rows f..f+7), f = 0..BX.
    // The scheme of each face (interface class, closure masks, scale) is
    // decided once here for all five components.
    const int flim = min(BX, (per ? n : n - 1) - i0);  // last slot needed
    for (int slot = t; slot <= BX; slot += BX) {
        const int jf = i0 - 1 + slot;
        uint8_t code = 0xff;
        R isc = (R)0;
        if (slot <= flim && (per || jf >= 0)) {
            int cm = 0;
#pragma unroll
            for (int o = 0; o < 8; ++o) cm = max(cm, (int)sc[slot + o]);
            int mp, mm;
            const int use = face_use(A.ph, per, n, jf, cm, &mp, &mm);
            code = (uint8_t)(use | (mp << 2) | (mm << 5));
            if (use) isc = face_iscale<R>(ss[slot + 3], ss[slot + 4]);
        }
        suse[slot] = code;
        sisc[slot] = isc;
    }
    __syncthreads();
    // A job is 4 consecutive faces of one component, computed from one
    // 12-value window per side (vector shared-memory loads).
    constexpr int NG = (BX + 1 + 3) / 4;
    for (int job = t; job < 5 * NG; job += BX) {
        const int q = job / NG, f0 = 4 * (job - q * NG);
        if (f0 > flim) continue;
        R pv[12], mv[12];
#pragma unroll
        for (int b = 0; b < 12; b += 16 / (int)sizeof(R)) {
            if constexpr (sizeof(R) == 4) {
                const float4 a = *reinterpret_cast<const float4*>(&sf[q][f0 + b]);
                const float4 c = *reinterpret_cast<const float4*>(&sf[5 + q][f0 + b]);
                pv[b] = (R)a.x; pv[b + 1] = (R)a.y; pv[b + 2] = (R)a.z; pv[b + 3] = (R)a.w;
                mv[b] = (R)c.x; mv[b + 1] = (R)c.y; mv[b + 2] = (R)c.z; mv[b + 3] = (R)c.w;
            } else {
                const double2 a = *reinterpret_cast<const double2*>(&sf[q][f0 + b]);
                const double2 c = *reinterpret_cast<const double2*>(&sf[5 + q][f0 + b]);
                pv[b] = (R)a.x; pv[b + 1] = (R)a.y;
                mv[b] = (R)c.x; mv[b + 1] = (R)c.y;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int slot = f0 + u;
            if (slot > BX) break;
            const int code = suse[slot];
            if (code == 0xff) continue;
            const int use = code & 3, mp = (code >> 2) & 7, mm = code >> 5;
            if (CHAR && use) continue;  // characteristic faces below
            const R isc = sisc[slot];
            R p8[8], m8[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                p8[o] = pv[u + o];
                m8[o] = mv[u + o];
            }
            sh[q][slot] = face_flux<R>(use, p8, m8, pk<R>(A.ph.eps, A.ph.epsf), isc, mp, mm);
        }
    }
    if constexpr (CHAR) {
        // WENO faces in characteristic variables: one thread per face, all
        // five components (slots other threads' jobs skipped above)
        for (int slot = t; slot <= BX; slot += BX) {
            const int code = suse[slot];
            if (code == 0xff || (code & 3) == 0) continue;
            const int jf = i0 - 1 + slot;
            const int ia = per ? wrapi(jf, n) : jf, ib = per ? wrapi(jf + 1, n) : jf + 1;
            R n1, n2, n3;
            face_normal<R>(g, 0, midx(g, ia, j, row + ia), midx(g, ib, j, row + ib), &n1, &n2, &n3);
            R out[5];
            face_flux_char<R>(A.ph, code & 3, pk<R>(A.ph.eps, A.ph.epsf), sisc[slot], (code >> 2) & 7, code >> 5,
                              A.U, g.N, row + ia, row + ib, n1, n2, n3,
                              [&](int o, int q) { return sf[q][slot + o]; },
                              [&](int o, int q) { return sf[5 + q][slot + o]; }, out);
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][slot] = out[q];
        }
    }
    __syncthreads();
    const int hi = per ? n : n - 1;
    int i = i0 + t;
    if (i < hi) {
        long long nn = row + i;
        R val[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) val[q] = -(sh[q][t + 1] - sh[q][t]);
        if (A.Fv) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                val[r + 1] += dvisc<R, P8>(A.ph.vorder, per, n, i, [&](int mm) { return sv[r][mm - (i0 - 4)]; });
        }
        epilogue<R, EP>(A, nn, i, j, k, val);
    }
    // zero the non-periodic boundary nodes of the accumulator
    if (EP == EP_STORE && !per && vb.x == 0 && t < 2) {
        int ib = t == 0 ? 0 : n - 1;
        R* Racc = (R*)A.R;
#pragma unroll
        for (int q = 0; q < 5; ++q) Racc[q * g.N + row + ib] = (R)0;
    }
}

// eta / zeta sweep: each warp owns 32 consecutive x of one line family and
// streams along the sweep direction, keeping the split fluxes of the last 8
// nodes in a per-lane shared-memory ring (every lane touches only its own
// column, so no synchronisation is needed).
template <class R, int DIR, int EP>
__global__ void __launch_bounds__(128) k_sweep_s(SweepArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo& g = A.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R* ring = reinterpret_cast<R*>(smem_raw) + (size_t)warp * (8 * 11 * 32);  // [8][f+, f-, sigma][32]
    const int nx = g.nx;
    const int n = DIR == 1 ? g.ny : g.nz;
    const int nother = DIR == 1 ? g.nz : g.ny;
    const long long stride = DIR == 1 ? (long long)nx : (long long)nx * g.ny;
    const int per = g.per[DIR];
    const int lo = per ? 0 : 1, hi = per ? n : n - 1;  // right-hand-side nodes [lo, hi)
    const int S = A.seg_len;
    const int nseg = (hi - lo + S - 1) / S;
    const int nxc = (nx + 31) / 32;
    const long long wid = (long long)blockIdx.x * 4 + warp;
    const int xc = (int)(wid % nxc);
    const long long rest = wid / nxc;
    const int o = (int)(rest % nother);
    const long long seg = rest / nother;
    if (seg >= nseg) return;
    const int i = xc * 32 + lane;
    const bool lane_ok = i < nx;
    const int m0 = lo + (int)seg * S;
    const int m1 = min(m0 + S, hi);
    // node (i, m, o): j = m, k = o (DIR 1) or j = o, k = m (DIR 2)
    const long long base = DIR == 1 ? (long long)i + (long long)nx * g.ny * o : (long long)i + (long long)nx * o;
    R fprev[5];
    unsigned long long cwin = 0ull;
    const int nsteps = (m1 - m0) + 8;
    for (int s = 0; s < nsteps; ++s) {
        const int m = m0 - 4 + s;
        const int slot = s & 7;
        R fp[5], fm[5], sg = (R)0;
        uint8_t c = 0;
        bool ok = lane_ok && (per || (m >= 0 && m < n));
        if (ok) ok = in_range(A.err, base + (long long)(per ? wrapi(m, n) : m) * stride, g.N);
        if (ok) {
            int mm = per ? wrapi(m, n) : m;
            long long nn = base + (long long)mm * stride;
            int jj = DIR == 1 ? mm : o;
            sg = node_split<R>(A, DIR, nn, i, jj, fp, fm);
            if (A.cls) c = A.cls[nn];
        } else {
#pragma unroll
            for (int q = 0; q < 5; ++q) fp[q] = fm[q] = (R)0;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            ring[(slot * 11 + q) * 32 + lane] = fp[q];
            ring[(slot * 11 + 5 + q) * 32 + lane] = fm[q];
        }
        ring[(slot * 11 + 10) * 32 + lane] = sg;
        cwin = (cwin << 8) | c;
        if (s >= 7) {
            const int jf = m - 4;  // face jf + 1/2 with nodes m-7 .. m
            int cm = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) cm = max(cm, (int)((cwin >> (8 * b)) & 0xff));
            int mp, mm;
            int use = face_use(A.ph, per, n, jf, cm, &mp, &mm);
            // nodes jf and jf+1 sit at window positions 3 and 4
            const R isc = use && lane_ok ? face_iscale<R>(ring[(((s - 4) & 7) * 11 + 10) * 32 + lane],
                                               ring[(((s - 3) & 7) * 11 + 10) * 32 + lane])
                              : (R)0;
            R fh[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                R p8[8], m8[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    int sl = (s - 7 + b) & 7;
                    p8[b] = ring[(sl * 11 + q) * 32 + lane];
                    m8[b] = ring[(sl * 11 + 5 + q) * 32 + lane];
                }
                fh[q] = face_flux<R>(use, p8, m8, pk<R>(A.ph.eps, A.ph.epsf), isc, mp, mm);
            }
            if (s >= 8 && lane_ok) {
                const int mn = m - 4;  // node
                const long long nn = base + (long long)mn * stride;
                R val[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) val[q] = -(fh[q] - fprev[q]);
                if (A.Fv) {
                    const long long lb = base;
                    visc_div<R>(A, DIR, lb, stride, n, mn, val);
                }
                const int jj = DIR == 1 ? mn : o, kk = DIR == 1 ? o : mn;
                epilogue<R, EP>(A, nn, i, jj, kk, val);
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) fprev[q] = fh[q];
        }
    }
}

// eta / zeta sweep on tiles: 32 consecutive x (lanes) by TL nodes along the
// sweep line plus a 4-node halo on each side.  The split fluxes and the
// viscous fluxes of the tile are staged in shared memory by all 8 warps at
// once (many loads in flight), faces are computed from shared memory, then
// differenced.  The halo costs 8/TL extra splits -- cheap in FP32, where the
// streaming form is latency-bound instead.
template <class R, int DIR, int EP, int TL, bool CHAR = false, bool P8 = false>
__device__ __forceinline__ void sweep_t_body(const SweepArgs& A, uint3 vb)
{
    constexpr int ROWS = TL + 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sf = reinterpret_cast<R*>(smem_raw);                      // [ROWS][10][32]
    R* sv = sf + (size_t)ROWS * 10 * 32;                          // [ROWS][4][32]
    uint8_t* sc = reinterpret_cast<uint8_t*>(sv + (size_t)ROWS * 4 * 32);  // [ROWS][32]
    const Geo& g = A.g;
    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int nx = g.nx;
    const int n = DIR == 1 ? g.ny : g.nz;
    const long long stride = DIR == 1 ? (long long)nx : (long long)nx * g.ny;
    const int per = g.per[DIR];
    const int lo = per ? 0 : 1, hi = per ? n : n - 1;
    const int i = vb.x * 32 + lane;
    const bool lane_ok = i < nx;
    const int o = vb.y;
    const int m0 = lo + vb.z * TL;
    const long long base = DIR == 1 ? (long long)i + (long long)nx * g.ny * o : (long long)i + (long long)nx * o;
    const long long N = g.N;
    const R* Fv = (const R*)A.Fv;
    // 0. the epilogue's operands of the tile's output nodes (the accumulator,
    //    and U, U^n for the RK update) are requested into L2 now, so that the
    //    epilogue at the end of the tile finds them there
    if (EP != EP_STORE && lane_ok) {
        for (int r = ty; r < TL; r += 8) {
            const int m = m0 + r;
            if (m >= hi) break;
            const long long nn = base + (long long)(per ? wrapi(m, n) : m) * stride;
            if (!in_range(A.err, nn, N)) break;
            prefetch_epilogue<R, EP>(A, nn);
        }
    }
    // 1. split fluxes, classes and viscous fluxes of the tile rows.  Every
    //    thread first issues the loads of all its rows (NR per warp), then
    //    splits: the loads of a tile are in flight together.
    constexpr int NR = (ROWS + 7) / 8;
    NodePrim<R> qv[NR];
    R fvv[NR][4];
    uint8_t cv[NR];
    bool okv[NR];
    long long miv[NR];
#pragma unroll
    for (int it = 0; it < NR; ++it) {
        const int r = ty + 8 * it;
        const int m = m0 - 4 + r;
        okv[it] = r < ROWS && lane_ok && (per || (m >= 0 && m < n));
        if (okv[it]) okv[it] = in_range(A.err, base + (long long)(per ? wrapi(m, n) : m) * stride, N);
        cv[it] = 0;
        miv[it] = 0;
        if (okv[it]) {
            const int mm = per ? wrapi(m, n) : m;
            const long long nn = base + (long long)mm * stride;
            miv[it] = midx(g, i, DIR == 1 ? mm : o, nn);
            qv[it] = load_prim<R>(A, nn);
            if (A.cls) cv[it] = __ldg(A.cls + nn);
            if (Fv) {
#pragma unroll
                for (int row = 0; row < 4; ++row) fvv[it][row] = __ldg(Fv + (long long)(4 * DIR + row) * N + nn);
            }
        }
    }
#pragma unroll
    for (int it = 0; it < NR; ++it) {
        const int r = ty + 8 * it;
        if (r >= ROWS) break;
        R fp[5], fm[5];
        if (okv[it]) {
            split_prim<R>(A, DIR, qv[it], miv[it], fp, fm);
        } else {
#pragma unroll
            for (int q = 0; q < 5; ++q) fp[q] = fm[q] = (R)0;
        }
        if (Fv) {
#pragma unroll
            for (int row = 0; row < 4; ++row) sv[(r * 4 + row) * 32 + lane] = okv[it] ? fvv[it][row] : (R)0;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            sf[(r * 10 + q) * 32 + lane] = fp[q];
            sf[(r * 10 + 5 + q) * 32 + lane] = fm[q];
        }
        sc[r * 32 + lane] = cv[it];
    }
    __syncthreads();
    // 2. faces (m0-1+f)+1/2, f = 0..TL, from rows f..f+7.  Thread row ty
    //    owns FPT consecutive faces and reads their FPT+7 rows once per
    //    component; results stay in registers until the buffer is reused.
    constexpr int FPT = (TL + 1 + 7) / 8;
    constexpr int WIN = FPT + 7;
    const int fbase = ty * FPT;
    R fh[FPT][5], iscv[FPT];
    int usev[FPT], mpv[FPT], mmv[FPT];
#pragma unroll
    for (int u = 0; u < FPT; ++u) {
        const int f = fbase + u;
        const int jf = m0 - 1 + f;
        usev[u] = -1;
        iscv[u] = (R)0;
        if (f > TL || !(per || (jf >= 0 && jf <= n - 2))) continue;
        int cm = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) cm = max(cm, (int)sc[(f + b) * 32 + lane]);
        usev[u] = face_use(A.ph, per, n, jf, cm, &mpv[u], &mmv[u]);
        if (usev[u] > 0 && lane_ok) {
            // sigma of nodes jf and jf+1 from the metrics (WENO faces only)
            const int ma = per ? wrapi(jf, n) : jf, mb = per ? wrapi(jf + 1, n) : jf + 1;
            const long long na = base + (long long)ma * stride, nb = base + (long long)mb * stride;
            iscv[u] = face_iscale<R>(metr<R>(g, M_SIG + DIR, midx(g, i, DIR == 1 ? ma : o, na)),
                                     metr<R>(g, M_SIG + DIR, midx(g, i, DIR == 1 ? mb : o, nb)));
        }
    }
    if constexpr (CHAR) {
        // WENO faces in characteristic variables (all five components)
#pragma unroll
        for (int u = 0; u < FPT; ++u) {
            if (usev[u] <= 0) continue;
            if (!lane_ok) {
#pragma unroll
                for (int q = 0; q < 5; ++q) fh[u][q] = (R)0;
                continue;
            }
            const int f = fbase + u, jf = m0 - 1 + f;
            const int ma = per ? wrapi(jf, n) : jf, mb = per ? wrapi(jf + 1, n) : jf + 1;
            const long long na = base + (long long)ma * stride, nb = base + (long long)mb * stride;
            R n1, n2, n3;
            face_normal<R>(g, DIR, midx(g, i, DIR == 1 ? ma : o, na), midx(g, i, DIR == 1 ? mb : o, nb), &n1, &n2,
                           &n3);
            face_flux_char<R>(A.ph, usev[u], pk<R>(A.ph.eps, A.ph.epsf), iscv[u], mpv[u], mmv[u], A.U, N, na, nb,
                              n1, n2, n3, [&](int b, int q) { return sf[((f + b) * 10 + q) * 32 + lane]; },
                              [&](int b, int q) { return sf[((f + b) * 10 + 5 + q) * 32 + lane]; }, fh[u]);
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        R pv[WIN], mv[WIN];
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            const int r = min(fbase + b, ROWS - 1);
            pv[b] = sf[(r * 10 + q) * 32 + lane];
            mv[b] = sf[(r * 10 + 5 + q) * 32 + lane];
        }
#pragma unroll
        for (int u = 0; u < FPT; ++u) {
            if (usev[u] < 0) {
                fh[u][q] = (R)0;
                continue;
            }
            if (CHAR && usev[u] > 0) continue;  // done above
            R p8[8], m8[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                p8[b] = pv[u + b];
                m8[b] = mv[u + b];
            }
            fh[u][q] = face_flux<R>(usev[u], p8, m8, pk<R>(A.ph.eps, A.ph.epsf), iscv[u], mpv[u], mmv[u]);
        }
    }
    __syncthreads();
    R* sh = sf;  // faces reuse the split-flux buffer: [TL+1][5][32]
#pragma unroll
    for (int u = 0; u < FPT; ++u) {
        const int f = fbase + u;
        if (f > TL) break;
#pragma unroll
        for (int q = 0; q < 5; ++q) sh[(f * 5 + q) * 32 + lane] = fh[u][q];
    }
    __syncthreads();
    // 3. difference, viscous divergence and the epilogue
    for (int r = ty; r < TL && lane_ok; r += 8) {
        const int m = m0 + r;
        if (m >= hi) break;
        R val[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) val[q] = -(sh[((r + 1) * 5 + q) * 32 + lane] - sh[(r * 5 + q) * 32 + lane]);
        if (Fv) {
            const int rowbase = m0 - 4;  // line position of tile row 0
#pragma unroll
            for (int row = 0; row < 4; ++row)
                val[row + 1] += dvisc<R, P8>(A.ph.vorder, per, n, m,
                                                 [&](int mm) { return sv[((mm - rowbase) * 4 + row) * 32 + lane]; });
        }
        const int mm = per ? wrapi(m, n) : m;
        const long long nn = base + (long long)mm * stride;
        const int jj = DIR == 1 ? mm : o, kk = DIR == 1 ? o : mm;
        epilogue<R, EP>(A, nn, i, jj, kk, val);
    }
}

template <class R, int TL>
constexpr size_t tile_smem_bytes()
{
    return (size_t)(TL + 8) * 32 * (10 + 4) * sizeof(R) + (size_t)(TL + 8) * 32;
}

// ---------------------------------------------------------------------------
// walking sweeps: a CTA walks along its line segment in chunks and carries the
// split fluxes of the last eight stencil nodes and the last face value from
// one chunk to the next, so every node of the segment is split once and every
// face is reconstructed once (the tiles above split their 8-node halos again
// in every tile).  Same operations, in the same order per face and node, as
// the tiled sweeps: the results are bit-identical.
// ---------------------------------------------------------------------------

// split fluxes (+ sigma, class, viscous fluxes of direction d) of line
// position m of a line, or zeros outside a non-periodic line
template <class R>
struct RowVals {
    R fp[5], fm[5], sg, fv[4];
    uint8_t c;
    bool ok;
};

template <class R, int DIR>
__device__ __forceinline__ void row_vals(const SweepArgs& A, long long base, long long stride, int n, int per, int m,
                                         int i, int o, bool lane_ok, RowVals<R>& r)
{
    const Geo& g = A.g;
    r.ok = lane_ok && (per || (m >= 0 && m < n));
    const int mm = per ? wrapi(m, n) : m;
    if (r.ok) r.ok = in_range(A.err, base + (long long)mm * stride, g.N);
    r.c = 0;
    if (r.ok) {
        const long long nn = base + (long long)mm * stride;
        const int jj = DIR == 0 ? o : (DIR == 1 ? mm : o);
        const int ii = DIR == 0 ? mm : i;
        r.sg = node_split<R>(A, DIR, nn, ii, jj, r.fp, r.fm);
        if (A.cls) r.c = __ldg(A.cls + nn);
        if (A.Fv) {
#pragma unroll
            for (int q = 0; q < 4; ++q) r.fv[q] = __ldg((const R*)A.Fv + (long long)(4 * DIR + q) * g.N + nn);
        }
    } else {
        r.sg = (R)0;
#pragma unroll
        for (int q = 0; q < 5; ++q) r.fp[q] = r.fm[q] = (R)0;
#pragma unroll
        for (int q = 0; q < 4; ++q) r.fv[q] = (R)0;
    }
}

// xi sweep, walking: one CTA of XW threads per segment of an x-line (j, k) =
// (vb.y, vb.z); segment vb.x covers right-hand-side nodes [ms, me) of the
// line in chunks of XW nodes.  Buffer row r holds line position m0 - 4 + r
// (r = 0..XW+7), face slot f holds face m0 - 1/2 + f (stencil rows f..f+7).
// Rows 0..7 and face slot 0 come from the previous chunk.  Rows are stored
// with an offset of 3 so that the four-face windows of slots 1+4g.. start on
// a 16-byte boundary.
constexpr int XW = 128;

template <class R, int EP>
__device__ __forceinline__ void sweep_xw_body(const SweepArgs& A, uint3 vb, int seg_len)
{
    constexpr int ROWS = XW + 8;
    constexpr int OFF = 3;
    __shared__ __align__(16) R sf[10][ROWS + OFF + 5];
    __shared__ R ss[ROWS];
    __shared__ R sv[4][ROWS];
    __shared__ uint8_t sc[ROWS];
    __shared__ R sh[5][XW + 1];
    __shared__ uint8_t suse[XW + 1];
    __shared__ R sisc[XW + 1];
    const Geo& g = A.g;
    const int n = g.nx;
    const int per = g.per[0];
    const int j = vb.y, k = vb.z;
    const int lo = per ? 0 : 1, hi = per ? n : n - 1;
    const int ms = lo + (int)vb.x * seg_len;
    if (ms >= hi) return;
    const int me = min(ms + seg_len, hi);
    const long long row = (long long)n * (j + (long long)g.ny * k);
    const int t = threadIdx.x;
    const R eps = pk<R>(A.ph.eps, A.ph.epsf);
    auto put_row = [&](int r, const RowVals<R>& v) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            sf[q][OFF + r] = v.fp[q];
            sf[5 + q][OFF + r] = v.fm[q];
        }
        ss[r] = v.sg;
        sc[r] = v.c;
#pragma unroll
        for (int q = 0; q < 4; ++q) sv[q][r] = v.fv[q];
    };
    // scheme of face slot f (face j = m0 - 1 + f)
    auto decide = [&](int m0, int f) {
        const int jf = m0 - 1 + f;
        uint8_t code = 0xff;
        R isc = (R)0;
        if (jf <= me - 1 && (per || jf >= 0)) {
            int cm = 0;
#pragma unroll
            for (int o = 0; o < 8; ++o) cm = max(cm, (int)sc[f + o]);
            int mp, mm;
            const int use = face_use(A.ph, per, n, jf, cm, &mp, &mm);
            code = (uint8_t)(use | (mp << 2) | (mm << 5));
            if (use) isc = face_iscale<R>(ss[f + 3], ss[f + 4]);
        }
        suse[f] = code;
        sisc[f] = isc;
    };
    auto one_face = [&](int f, int q) {
        const int code = suse[f];
        if (code == 0xff) return;
        R p8[8], m8[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            p8[o] = sf[q][OFF + f + o];
            m8[o] = sf[5 + q][OFF + f + o];
        }
        sh[q][f] = face_flux<R>(code & 3, p8, m8, eps, sisc[f], (code >> 2) & 7, code >> 5);
    };
    for (int m0 = ms; m0 < me; m0 += XW) {
        const bool first = m0 == ms;
        // the next chunk's new rows requested into L2
        {
            const int mr = m0 + XW + 4 + t;
            if (mr <= me + 3 && (per || mr < n)) {
                const long long nn = row + (per ? wrapi(mr, n) : mr);
                if (in_range(A.err, nn, g.N)) prefetch_row_inputs<R>(A, 0, nn);
            }
        }
        // new rows: line positions m0+4 .. m0+XW+3 (all XW+8 rows in the first
        // chunk); loaded and split before the barrier, stored after it
        RowVals<R> v, v2;
        {
            const int m = first ? m0 - 4 + t : m0 + 4 + t;
            if (m <= me + 3) row_vals<R, 0>(A, row, 1, n, per, m, 0, j, true, v);
            else v = RowVals<R>{};
            v2 = RowVals<R>{};
            if (first && t < 8 && m0 - 4 + XW + t <= me + 3)
                row_vals<R, 0>(A, row, 1, n, per, m0 - 4 + XW + t, 0, j, true, v2);
        }
        // carried values (rows XW..XW+7 and face slot XW of the previous chunk,
        // stable since that chunk's second barrier) into registers
        R cv = (R)0, hv = (R)0;
        uint8_t cc = 0;
        if (!first) {
            if (t < 8 * 15) {
                const int r = t & 7, e = t >> 3;
                cv = e < 10 ? sf[e][OFF + XW + r] : (e == 10 ? ss[XW + r] : sv[e - 11][XW + r]);
                if (e == 0) cc = sc[XW + r];
            }
            if (t < 5) hv = sh[t][XW];
        }
        __syncthreads();  // the previous chunk's faces and rows are consumed
        if (first) {
            put_row(t, v);
            if (t < 8) put_row(XW + t, v2);
        } else {
            if (t < 8 * 15) {
                const int r = t & 7, e = t >> 3;
                if (e < 10) sf[e][OFF + r] = cv;
                else if (e == 10) ss[r] = cv;
                else sv[e - 11][r] = cv;
                if (e == 0) sc[r] = cc;
            }
            if (t < 5) sh[t][0] = hv;
            put_row(8 + t, v);
        }
        __syncthreads();
        decide(m0, 1 + t);
        if (first && t == 0) decide(m0, 0);
        __syncthreads();
        // faces 1..XW: jobs of four consecutive faces of one component from one
        // twelve-value window per side (vector shared-memory loads)
        constexpr int NG = XW / 4;
        for (int job = t; job < 5 * NG; job += XW) {
            const int q = job / NG, f0 = 1 + 4 * (job - q * NG);
            if (m0 - 1 + f0 > me - 1) continue;
            R pv[12], mv[12];
#pragma unroll
            for (int b = 0; b < 12; b += 16 / (int)sizeof(R)) {
                if constexpr (sizeof(R) == 4) {
                    const float4 a = *reinterpret_cast<const float4*>(&sf[q][OFF + f0 + b]);
                    const float4 c = *reinterpret_cast<const float4*>(&sf[5 + q][OFF + f0 + b]);
                    pv[b] = (R)a.x; pv[b + 1] = (R)a.y; pv[b + 2] = (R)a.z; pv[b + 3] = (R)a.w;
                    mv[b] = (R)c.x; mv[b + 1] = (R)c.y; mv[b + 2] = (R)c.z; mv[b + 3] = (R)c.w;
                } else {
                    const double2 a = *reinterpret_cast<const double2*>(&sf[q][OFF + f0 + b]);
                    const double2 c = *reinterpret_cast<const double2*>(&sf[5 + q][OFF + f0 + b]);
                    pv[b] = (R)a.x; pv[b + 1] = (R)a.y;
                    mv[b] = (R)c.x; mv[b + 1] = (R)c.y;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + u;
                const int code = suse[f];
                if (code == 0xff) continue;
                R p8[8], m8[8];
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    p8[o] = pv[u + o];
                    m8[o] = mv[u + o];
                }
                sh[q][f] = face_flux<R>(code & 3, p8, m8, eps, sisc[f], (code >> 2) & 7, code >> 5);
            }
        }
        if (first && t < 5) one_face(0, t);
        __syncthreads();
        const int i = m0 + t;
        if (i < me) {
            R val[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) val[q] = -(sh[q][t + 1] - sh[q][t]);
            if (A.Fv) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    val[r + 1] += dcentral_tile<R>(A.ph.vorder, per, n, i, [&](int mm) { return sv[r][mm - (m0 - 4)]; });
            }
            epilogue<R, EP>(A, row + i, i, j, k, val);
        }
    }
    // zero the non-periodic boundary nodes of the accumulator
    if (EP == EP_STORE && !per && vb.x == 0 && t < 2) {
        const int ib = t == 0 ? 0 : n - 1;
        R* Racc = (R*)A.R;
#pragma unroll
        for (int q = 0; q < 5; ++q) Racc[q * g.N + row + ib] = (R)0;
    }
}

// eta / zeta sweep, walking: a CTA of 8 warps owns 32 consecutive x (lanes)
// of one line family (o = vb.y) and walks the right-hand-side nodes [ms, me)
// of segment vb.z in chunks of 8 line positions, one per warp.  Walk position
// q = m - (ms - 4); the split fluxes, sigma and classes of position q live in
// ring slot q & 15, the viscous fluxes in slot q & 31, face j + 1/2 in slot
// (j - ms + 1) & 15.  Per chunk: (A) each warp splits one new position,
// (B) each warp reconstructs one face, (C) each warp differences one node.
// The split ring is rewritten only after the barrier that ends (B), the
// viscous ring holds the 24 positions a chunk's (C) and the next chunk's (A)
// touch, and the face ring is rewritten only after the next chunk's first
// barrier -- two barriers per chunk.
constexpr int WS_RING = 16, WV_RING = 32;

template <class R>
constexpr size_t walk_smem_bytes()
{
    return (size_t)WS_RING * 11 * 32 * sizeof(R) + (size_t)WV_RING * 4 * 32 * sizeof(R) +
           (size_t)WS_RING * 5 * 32 * sizeof(R) + (size_t)WS_RING * 32;
}

template <class R, int DIR, int EP, bool P8 = false>
__device__ __forceinline__ void sweep_w_body(const SweepArgs& A, uint3 vb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sf = reinterpret_cast<R*>(smem_raw);       // [16][10][32] f+, f-
    R* ss = sf + WS_RING * 10 * 32;               // [16][32] sigma
    R* sv = ss + WS_RING * 32;                    // [32][4][32] viscous fluxes of DIR
    R* sh = sv + WV_RING * 4 * 32;                // [16][5][32] faces
    uint8_t* sc = reinterpret_cast<uint8_t*>(sh + WS_RING * 5 * 32);  // [16][32]
    const Geo& g = A.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nx = g.nx;
    const int n = DIR == 1 ? g.ny : g.nz;
    const long long stride = DIR == 1 ? (long long)nx : (long long)nx * g.ny;
    const int per = g.per[DIR];
    const int lo = per ? 0 : 1, hi = per ? n : n - 1;
    const int i = vb.x * 32 + lane;
    const bool lane_ok = i < nx;
    const int o = vb.y;
    const int S = A.seg_len;
    const int ms = lo + (int)vb.z * S;
    if (ms >= hi) return;
    const int me = min(ms + S, hi);
    const long long base = DIR == 1 ? (long long)i + (long long)nx * g.ny * o : (long long)i + (long long)nx * o;
    const R eps = pk<R>(A.ph.eps, A.ph.epsf);
    auto load_row = [&](int m) {
        const int q = m - (ms - 4);
        RowVals<R> v;
        row_vals<R, DIR>(A, base, stride, n, per, m, i, o, lane_ok, v);
        R* f = sf + (size_t)(q & (WS_RING - 1)) * 10 * 32 + lane;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            f[c * 32] = v.fp[c];
            f[(5 + c) * 32] = v.fm[c];
        }
        ss[(q & (WS_RING - 1)) * 32 + lane] = v.sg;
        sc[(q & (WS_RING - 1)) * 32 + lane] = v.c;
        if (A.Fv) {
#pragma unroll
            for (int c = 0; c < 4; ++c) sv[((q & (WV_RING - 1)) * 4 + c) * 32 + lane] = v.fv[c];
        }
    };
    // face jf + 1/2 from ring rows q(jf-3) .. q(jf+4)
    auto face = [&](int jf) {
        const int q0 = jf - 3 - (ms - 4);
        int cm = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) cm = max(cm, (int)sc[((q0 + b) & (WS_RING - 1)) * 32 + lane]);
        int mp, mm;
        const int use = face_use(A.ph, per, n, jf, cm, &mp, &mm);
        const R isc = use && lane_ok ? face_iscale<R>(ss[((q0 + 3) & (WS_RING - 1)) * 32 + lane],
                                                      ss[((q0 + 4) & (WS_RING - 1)) * 32 + lane])
                                     : (R)0;
        R* out = sh + (size_t)((jf - ms + 1) & (WS_RING - 1)) * 5 * 32 + lane;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            R p8[8], m8[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const R* f = sf + (size_t)((q0 + b) & (WS_RING - 1)) * 10 * 32 + lane;
                p8[b] = f[c * 32];
                m8[b] = f[(5 + c) * 32];
            }
            out[c * 32] = face_flux<R>(use, p8, m8, eps, isc, mp, mm);
        }
    };
    // prologue: positions ms-4 .. ms+3 and the face ms - 1/2
    load_row(ms - 4 + w);
    __syncthreads();
    if (w == 0) face(ms - 1);
    for (int m0 = ms; m0 < me; m0 += 8) {
        // the next chunk's new position and output node requested into L2
        if (lane_ok) {
            const int mr = m0 + 12 + w, mo = m0 + 8 + w;
            if (mr <= me + 3 && (per || mr < n)) {
                const long long nn = base + (long long)(per ? wrapi(mr, n) : mr) * stride;
                if (in_range(A.err, nn, g.N)) prefetch_row_inputs<R>(A, DIR, nn);
            }
            if (mo < me) {
                const long long nn = base + (long long)(per ? wrapi(mo, n) : mo) * stride;
                if (in_range(A.err, nn, g.N)) prefetch_epilogue<R, EP>(A, nn);
            }
        }
        // (A) the new position m0 + 4 + w (needed up to me + 3)
        if (m0 + 4 + w <= me + 3) load_row(m0 + 4 + w);
        __syncthreads();
        // (B) face m0 + w + 1/2
        if (m0 + w <= me - 1) face(m0 + w);
        __syncthreads();
        // (C) node m0 + w
        const int m = m0 + w;
        if (m < me && lane_ok) {
            const R* f0 = sh + (size_t)((m - ms) & (WS_RING - 1)) * 5 * 32 + lane;
            const R* f1 = sh + (size_t)((m - ms + 1) & (WS_RING - 1)) * 5 * 32 + lane;
            R val[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) val[c] = -(f1[c * 32] - f0[c * 32]);
            if (A.Fv) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    val[c + 1] += dvisc<R, P8>(A.ph.vorder, per, n, m, [&](int mm) {
                        return sv[(((mm - (ms - 4)) & (WV_RING - 1)) * 4 + c) * 32 + lane];
                    });
            }
            const int mm = per ? wrapi(m, n) : m;
            const long long nn = base + (long long)mm * stride;
            const int jj = DIR == 1 ? mm : o, kk = DIR == 1 ? o : mm;
            epilogue<R, EP>(A, nn, i, jj, kk, val);
        }
    }
}

// dynamic shared memory of k_sweep_s: 4 warps x 8 ring slots x 11 values x 32 lanes
template <class R>
constexpr size_t stream_smem_bytes()
{
    return (size_t)4 * 8 * 11 * 32 * sizeof(R);
}

// ---------------------------------------------------------------------------
// TMA-staged walking eta / zeta sweep (FP32-bulk form).  The same walk and the
// same arithmetic as sweep_w_body, but the rows a chunk splits are fetched by
// the tensor-memory accelerator (cp.async.bulk.tensor, one 32-node row of a
// field per copy) into a ring of NBUF staging buffers, NBUF - 1 row groups
// ahead of the warps that split them; completion is signalled on one mbarrier
// per buffer.  The node operands of the epilogue (R; U and U^n in the RK
// variant) are loaded into registers one chunk ahead.  Every wait is bounded:
// a wait that gives up sets the flag 8 (bit 3) of the error word, the block waits (again
// bounded) for the copies it issued and returns.
// ---------------------------------------------------------------------------
struct TmaRowMaps {
    CUtensorMap p4;   // P as [7][nz][ny][nx] float, box 32 x 1 x 1 x 4 (rho, u, v, w)
    CUtensorMap p1;   // the same tensor, box 32 x 1 x 1 x 1 (c)
    CUtensorMap fv;   // Fv as [12][nz][ny][nx] float, box 32 x 1 x 1 x 4
    CUtensorMap cls;  // classes as [nz][ny][nx] uint8, box 32 x 1 x 1
};

// staging layout of one row (bytes): P rho,u,v,w [4][32] at 0, c [32] at
// 512, Fv [4][32] at 640, classes [32] at 1152; 1280 per row, 8 rows a group
constexpr int TW_NBUF = 4, TW_ROW = 1280, TW_GROUP = 8 * TW_ROW;

constexpr size_t walk_tma_smem_bytes()
{
    return (size_t)TW_NBUF * TW_GROUP + walk_smem_bytes<float>() + 64;  // + mbarriers and the abort flag
}

template <int DIR, int EP>
__device__ __forceinline__ void sweep_wt_body(const SweepArgs& A, const TmaRowMaps& maps, uint3 vb)
{
    using R = float;
    extern __shared__ __align__(128) unsigned char smem_tw[];
    unsigned char* stage = smem_tw;                                    // [NBUF][8][1280]
    R* sf = reinterpret_cast<R*>(smem_tw + TW_NBUF * TW_GROUP);         // rings as in sweep_w_body
    R* ss = sf + WS_RING * 10 * 32;
    R* sv = ss + WS_RING * 32;
    R* sh = sv + WV_RING * 4 * 32;
    uint8_t* sc = reinterpret_cast<uint8_t*>(sh + WS_RING * 5 * 32);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sc + WS_RING * 32);   // [NBUF]
    int& s_abort = *reinterpret_cast<int*>(bars + TW_NBUF);
    const Geo& g = A.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nx = g.nx;
    const int n = DIR == 1 ? g.ny : g.nz;
    const long long stride = DIR == 1 ? (long long)nx : (long long)nx * g.ny;
    const int per = g.per[DIR];
    const int lo = per ? 0 : 1, hi = per ? n : n - 1;
    const int x0 = vb.x * 32;
    const int i = x0 + lane;
    const bool lane_ok = i < nx;
    const int o = vb.y;
    const int S = A.seg_len;
    const int ms = lo + (int)vb.z * S;
    if (ms >= hi) return;
    const int me = min(ms + S, hi);
    const long long base = DIR == 1 ? (long long)i + (long long)nx * g.ny * o : (long long)i + (long long)nx * o;
    const R eps = pk<R>(A.ph.eps, A.ph.epsf);
    // row groups: group gi holds walk positions q = 8 gi .. 8 gi + 7 (line
    // positions ms - 4 + q); positions beyond me + 3 are never needed
    const int ngroups = (me + 3 - (ms - 4)) / 8 + 1;
    if (threadIdx.x == 0) {
        for (int b = 0; b < TW_NBUF; ++b) mbar_init(&bars[b], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto row_valid = [&](int m) { return (per || (m >= 0 && m < n)) && m <= me + 3; };
    // warp 0 issues the copies of group gi into buffer gi % NBUF: lane 4 r + t
    // copies piece t of row r (t: 0 rho..w, 1 c, 2 viscous fluxes, 3 classes)
    auto issue = [&](int gi) {
        if (gi >= ngroups) return;
        uint64_t* bar = &bars[gi % TW_NBUF];
        unsigned bytes = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (row_valid(ms - 4 + 8 * gi + r)) bytes += 640u + (A.Fv ? 512u : 0u) + (A.cls ? 32u : 0u);
        if (lane == 0) {
            if (bytes) mbar_arrive_expect_tx(bar, bytes);
            else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
        }
        __syncwarp();
        const int r = lane >> 2, t = lane & 3;
        const int m = ms - 4 + 8 * gi + r;
        if (!row_valid(m)) return;
        const int mm = per ? wrapi(m, n) : m;
        const int cy = DIR == 1 ? mm : o, cz = DIR == 1 ? o : mm;
        unsigned char* dst = stage + (size_t)(gi % TW_NBUF) * TW_GROUP + (size_t)r * TW_ROW;
        if (t == 0) tma_load_4d(dst, &maps.p4, x0, cy, cz, 0, bar);
        else if (t == 1) tma_load_4d(dst + 512, &maps.p1, x0, cy, cz, 6, bar);
        else if (t == 2) { if (A.Fv) tma_load_4d(dst + 640, &maps.fv, x0, cy, cz, 4 * DIR, bar); }
        else if (A.cls) tma_load_3d(dst + 1152, &maps.cls, x0, cy, cz, bar);
    };
    // wait for group gi; on a timeout every thread learns it at the next barrier
    auto wait_group = [&](int gi) {
        if (!mbar_wait_bounded(&bars[gi % TW_NBUF], (unsigned)((gi / TW_NBUF) & 1), TW_WAIT_LIMIT)) {
            atomicOr(A.err, 8);
            s_abort = 1;
        }
    };
    // drain: wait (bounded) for every group issued and not yet consumed
    auto drain = [&](int first_unconsumed, int last_issued) {
        if (threadIdx.x == 0)
            for (int gi = first_unconsumed; gi <= last_issued && gi < ngroups; ++gi)
                mbar_wait_bounded(&bars[gi % TW_NBUF], (unsigned)((gi / TW_NBUF) & 1), TW_WAIT_LIMIT);
        __syncthreads();
    };
    // split the row of group gi that this warp owns into the rings
    auto split_row = [&](int gi) {
        const int m = ms - 4 + 8 * gi + w;
        const int q = 8 * gi + w;
        const unsigned char* src = stage + (size_t)(gi % TW_NBUF) * TW_GROUP + (size_t)w * TW_ROW;
        const R* sp = reinterpret_cast<const R*>(src);
        R fp[5], fm[5], sg = (R)0, fvv[4] = {(R)0, (R)0, (R)0, (R)0};
        uint8_t c = 0;
        bool ok = lane_ok && row_valid(m);
        const int mm = per ? wrapi(m, n) : m;
        if (ok) ok = in_range(A.err, base + (long long)mm * stride, g.N);
        if (ok) {
            const long long nn = base + (long long)mm * stride;
            const long long mi = midx(g, i, DIR == 1 ? mm : o, nn);
            NodePrim<R> pr{sp[lane], sp[32 + lane], sp[64 + lane], sp[96 + lane], sp[128 + lane]};
            sg = split_prim<R>(A, DIR, pr, mi, fp, fm);
            if (A.cls) c = src[1152 + lane];
            if (A.Fv) {
#pragma unroll
                for (int e = 0; e < 4; ++e) fvv[e] = sp[160 + 32 * e + lane];
            }
        } else {
#pragma unroll
            for (int e = 0; e < 5; ++e) fp[e] = fm[e] = (R)0;
        }
        R* f = sf + (size_t)(q & (WS_RING - 1)) * 10 * 32 + lane;
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            f[e * 32] = fp[e];
            f[(5 + e) * 32] = fm[e];
        }
        ss[(q & (WS_RING - 1)) * 32 + lane] = sg;
        sc[(q & (WS_RING - 1)) * 32 + lane] = c;
        if (A.Fv) {
#pragma unroll
            for (int e = 0; e < 4; ++e) sv[((q & (WV_RING - 1)) * 4 + e) * 32 + lane] = fvv[e];
        }
    };
    auto face = [&](int jf) {
        const int q0 = jf - 3 - (ms - 4);
        int cm = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) cm = max(cm, (int)sc[((q0 + b) & (WS_RING - 1)) * 32 + lane]);
        int mp, mm;
        const int use = face_use(A.ph, per, n, jf, cm, &mp, &mm);
        const R isc = use && lane_ok ? face_iscale<R>(ss[((q0 + 3) & (WS_RING - 1)) * 32 + lane],
                                                      ss[((q0 + 4) & (WS_RING - 1)) * 32 + lane])
                                     : (R)0;
        R* out = sh + (size_t)((jf - ms + 1) & (WS_RING - 1)) * 5 * 32 + lane;
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            R p8[8], m8[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const R* f = sf + (size_t)((q0 + b) & (WS_RING - 1)) * 10 * 32 + lane;
                p8[b] = f[e * 32];
                m8[b] = f[(5 + e) * 32];
            }
            out[e * 32] = face_flux<R>(use, p8, m8, eps, isc, mp, mm);
        }
    };
    // epilogue operands of node m (R; U, U^n for the RK variant), in registers
    struct NodeOps {
        R r[5];
        double u[5], un[5];
    };
    auto load_ops = [&](int m, NodeOps& op) {
        if (!(m < me && lane_ok)) return;
        const int mm = per ? wrapi(m, n) : m;
        const long long nn = base + (long long)mm * stride;
        if (!in_range(A.err, nn, g.N)) return;
        const long long N = g.N;
        if (EP == EP_ACCUM || EP == EP_FINAL_RK || EP == EP_FINAL_RHS) {
#pragma unroll
            for (int e = 0; e < 5; ++e) op.r[e] = ((const R*)A.R)[e * N + nn];
        }
        if (EP == EP_FINAL_RK) {
            const bool bnd = is_bnd(g, i, DIR == 1 ? mm : o, DIR == 1 ? o : mm);
            if (!bnd) {
#pragma unroll
                for (int e = 0; e < 5; ++e) {
                    op.u[e] = A.U[e * N + nn];
                    op.un[e] = A.rk_a != 0.0 ? A.Un[e * N + nn] : 0.0;
                }
            }
        }
    };
    // the epilogue of sweep_w_body on preloaded operands
    auto finish = [&](int m, const R val[5], const NodeOps& op) {
        const int mm = per ? wrapi(m, n) : m;
        const long long nn = base + (long long)mm * stride;
        if (!in_range(A.err, nn, g.N)) return;
        const long long N = g.N;
        const int jj = DIR == 1 ? mm : o, kk = DIR == 1 ? o : mm;
        R* Racc = (R*)A.R;
        if (EP == EP_ACCUM) {
#pragma unroll
            for (int e = 0; e < 5; ++e) Racc[e * N + nn] = op.r[e] + val[e];
        } else {
            const bool bnd = is_bnd(g, i, jj, kk);
            const double J = metv(g, M_J, midx(g, i, jj, nn));
            if (EP == EP_FINAL_RHS) {
#pragma unroll
                for (int e = 0; e < 5; ++e) A.Lout[e * N + nn] = bnd ? 0.0 : J * to_f64(op.r[e] + val[e]);
            } else {
                if (bnd) return;
                const double dtJ = *A.dt * J;
#pragma unroll
                for (int e = 0; e < 5; ++e)
                    A.Uout[e * N + nn] = rk_combine(A, dtJ, to_f64(op.r[e] + val[e]), op.u[e], op.un[e]);
            }
        }
    };

    // prologue: groups 0 .. NBUF-1 in flight, group 0 split, face ms - 1/2
    if (w == 0)
        for (int gi = 0; gi < TW_NBUF; ++gi) issue(gi);
    NodeOps ops;
    load_ops(ms + w, ops);
    wait_group(0);
    __syncthreads();
    if (s_abort) { drain(0, TW_NBUF - 1); return; }
    split_row(0);
    __syncthreads();
    if (w == 0) issue(TW_NBUF);  // buffer 0 is free again
    if (w == 0) face(ms - 1);
    int gi = 1;
    for (int m0 = ms; m0 < me; m0 += 8, ++gi) {
        NodeOps next;
        load_ops(m0 + 8 + w, next);  // operands of the next chunk's node, in flight during this chunk
        // (A) the positions m0+4 .. m0+11 (group gi)
        if (gi < ngroups) wait_group(gi);
        __syncthreads();
        if (s_abort) { drain(gi, gi + TW_NBUF - 1); return; }
        if (gi < ngroups) split_row(gi);
        __syncthreads();
        if (w == 0) issue(gi + TW_NBUF);  // group gi's buffer is consumed
        // (B) face m0 + w + 1/2
        if (m0 + w <= me - 1) face(m0 + w);
        __syncthreads();
        // (C) node m0 + w
        const int m = m0 + w;
        if (m < me && lane_ok) {
            const R* f0 = sh + (size_t)((m - ms) & (WS_RING - 1)) * 5 * 32 + lane;
            const R* f1 = sh + (size_t)((m - ms + 1) & (WS_RING - 1)) * 5 * 32 + lane;
            R val[5];
#pragma unroll
            for (int e = 0; e < 5; ++e) val[e] = -(f1[e * 32] - f0[e * 32]);
            if (A.Fv) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    val[e + 1] += dcentral_tile<R>(A.ph.vorder, per, n, m, [&](int mq) {
                        return sv[(((mq - (ms - 4)) & (WV_RING - 1)) * 4 + e) * 32 + lane];
                    });
            }
            finish(m, val, ops);
        }
        ops = next;
    }
}

// ---------------------------------------------------------------------------
// Free-stream-preserving metric mode (reading R17; periodic lines): the
// metric vector of interface j+1/2 is the 8-point midpoint interpolation of
// the nodal alpha = grad(d)/J over nodes j-3 .. j+4, and all eight stencil
// nodes are split with that one frozen vector (so a uniform state gives the
// same split flux at every stencil node and the flux difference telescopes);
// the WENO indicators are scaled by its norm.  One thread per node computes
// both of its faces -- a test and robustness mode, not tuned for speed.
// ---------------------------------------------------------------------------
// Lagrange weights of the polynomial through offsets -3 .. 4 evaluated at 1/2
__device__ __forceinline__ double midpoint_weight(int l)
{
    double w = 1.0;
    for (int q = 0; q < 8; ++q)
        if (q != l) w *= (0.5 - (double)(q - 3)) / (double)(l - q);
    return w;
}

template <class R, int DIR>
__device__ __forceinline__ void fsp_face(const SweepArgs& A, long long base, long long stride, int n, int jf, int i,
                                         int o, R out[5])
{
    const Geo& g = A.g;
    R ai[3] = {(R)0, (R)0, (R)0};
    long long nn[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        const int mm = wrapi(jf - 3 + l, n);
        nn[l] = base + (long long)mm * stride;
        const long long mi = midx(g, DIR == 0 ? mm : i, DIR == 1 ? mm : o, nn[l]);
        const R w = (R)midpoint_weight(l);
#pragma unroll
        for (int e = 0; e < 3; ++e) ai[e] = mad(w, metr<R>(g, M_ALPHA + 3 * DIR + e, mi), ai[e]);
    }
    const R sig = sqrt(mad(ai[2], ai[2], mad(ai[1], ai[1], ai[0] * ai[0])));
    const R k1 = ai[0] / sig, k2 = ai[1] / sig, k3 = ai[2] / sig;
    R fp8[5][8], fm8[5][8];
    int cm = 0;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        const NodePrim<R> q = load_prim<R>(A, nn[l]);
        R fp[5], fm[5];
        sw_split<R>(A.ph, q.rho, q.u, q.v, q.w, q.c, k1, k2, k3, sig, fp, fm);
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            fp8[e][l] = fp[e];
            fm8[e][l] = fm[e];
        }
        if (A.cls) cm = max(cm, (int)A.cls[nn[l]]);
    }
    int mp, mm;
    const int use = face_use(A.ph, 1, n, jf, cm, &mp, &mm);
    const R isc = (R)1 / (sig * sig);
#pragma unroll
    for (int e = 0; e < 5; ++e) out[e] = face_flux<R>(use, fp8[e], fm8[e], pk<R>(A.ph.eps, A.ph.epsf), isc, 0, 0);
}

template <class R, int DIR, int EP>
__global__ void __launch_bounds__(128) k_sweep_fsp(SweepArgs A)
{
    const Geo& g = A.g;
    const uint3 vb = blockIdx;
    NODE_IJK(g)
    {
        const int pos[3] = {i, j, k};
        const int len = DIR == 0 ? g.nx : (DIR == 1 ? g.ny : g.nz);
        const long long stride = DIR == 0 ? 1 : (DIR == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
        const int m = pos[DIR];
        const long long base = n - (long long)m * stride;  // node 0 of this line
        R fl[5], fr[5];
        // metric index of a line node: (m, j) for xi, (i, m) for eta, (i, j) for zeta
        fsp_face<R, DIR>(A, base, stride, len, m - 1, i, j, fl);
        fsp_face<R, DIR>(A, base, stride, len, m, i, j, fr);
        R val[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) val[e] = -(fr[e] - fl[e]);
        if (A.Fv) {
            const R* Fv = (const R*)A.Fv;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const R* f = Fv + (long long)(4 * DIR + r) * g.N + base;
                val[r + 1] += dcentral<R>(A.ph.vorder, 1, len, m, [&](int q) { return __ldg(f + (long long)q * stride); });
            }
        }
        epilogue<R, EP>(A, n, i, j, k, val);
    }
}

// ---------------------------------------------------------------------------
// boundary conditions on the conserved state (reading R12), one direction per
// launch, faces lo and hi; applied in the order xi, eta, zeta.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cons_prim(const Phys& ph, const double* U, long long N, long long n, double o[5])
{
    double rho = U[n];
    double u = U[N + n] / rho, v = U[2 * N + n] / rho, w = U[3 * N + n] / rho;
    double p = ph.gm1 * (U[4 * N + n] - 0.5 * rho * (u * u + v * v + w * w));
    o[0] = rho; o[1] = u; o[2] = v; o[3] = w; o[4] = p;
}

__device__ __forceinline__ void put_prim(const Phys& ph, double* U, long long N, long long n, double rho, double u,
                                         double v, double w, double p)
{
    U[n] = rho;
    U[N + n] = rho * u;
    U[2 * N + n] = rho * v;
    U[3 * N + n] = rho * w;
    U[4 * N + n] = p * ph.inv_gm1 + 0.5 * rho * (u * u + v * v + w * w);
}

// ---------------------------------------------------------------------------
// multi-block halo exchange: ghost layers of one face of a block receive
// H layers of the neighbouring block's interior, all five conserved fields.
// One CTA row (blockIdx.y) per link of direction d.
// ---------------------------------------------------------------------------
struct HaloLink {
    double* dst;
    const double* src;
    long long dstN, srcN;
    int dnx, dny, snx, sny;  // node index = i + nx (j + ny k) in each grid
    int dl0, sl0;            // first layer along d in the destination / source
    int na, nb;              // extents in the directions (d+1)%3, (d+2)%3
};

__global__ void k_halo(const HaloLink* __restrict__ links, int d, int H)
{
    const HaloLink L = links[blockIdx.y];
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    const long long plane = (long long)L.na * L.nb;
    const long long per_field = (long long)H * plane;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 5 * per_field;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / per_field);
        const long long r = e - q * per_field;
        const int l = (int)(r / plane);
        const long long t = r - l * plane;
        int pd[3], ps[3];
        pd[a] = ps[a] = (int)(t % L.na);
        pd[b] = ps[b] = (int)(t / L.na);
        pd[d] = L.dl0 + l;
        ps[d] = L.sl0 + l;
        const long long nd = pd[0] + (long long)L.dnx * (pd[1] + (long long)L.dny * pd[2]);
        const long long ns = ps[0] + (long long)L.snx * (ps[1] + (long long)L.sny * ps[2]);
        L.dst[q * L.dstN + nd] = L.src[q * L.srcN + ns];
    }
}

// state copy between device memory and pinned (device-mapped) host memory
// by the SMs: 16-byte loads and stores over the CPU-GPU link, many in flight
// (n2: number of double2 items; a trailing odd double is copied by thread 0)
__global__ void k_copy_mapped(double2* __restrict__ dst, const double2* __restrict__ src, long long n2, double* dst1,
                              const double* src1, int odd)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2; e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e];
    if (odd && blockIdx.x == 0 && threadIdx.x == 0) *dst1 = *src1;
}

// Non-reflecting boundary node n (neighbour n1 one node inward), outward
// normal along sgn * grad(d) of the metrics at the node: the characteristic
// changes toward the interior -- entropy dp - c^2 drho, shear dv - (dv.n)n,
// acoustic dp +- rho c dv_n with speeds u_n, u_n, u_n +- c -- are taken where
// the speed is positive (the wave leaves) and dropped where it enters
// (Thompson 1987, as an update of the boundary node).
__device__ __forceinline__ void nonreflect_node(const Geo& g, const Phys& ph, double* U, long long n, long long n1,
                                                int i, int j, int d, double sgn)
{
    const long long N = g.N;
    double ob[5], o1[5];
    cons_prim(ph, U, N, n, ob);
    cons_prim(ph, U, N, n1, o1);
    const long long mi = midx(g, i, j, n);
    const double g0 = metv(g, 3 * d, mi), g1 = metv(g, 3 * d + 1, mi), g2 = metv(g, 3 * d + 2, mi);
    const double gn = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    const double nx = sgn * g0 / gn, ny = sgn * g1 / gn, nz = sgn * g2 / gn;
    const double rho = ob[0], c = sqrt(ph.gamma * ob[4] / ob[0]);
    const double un = ob[1] * nx + ob[2] * ny + ob[3] * nz;
    const double drho = o1[0] - ob[0], du = o1[1] - ob[1], dv = o1[2] - ob[2], dw = o1[3] - ob[3];
    const double dp = o1[4] - ob[4];
    const double dvn = du * nx + dv * ny + dw * nz;
    double e_ent = dp - c * c * drho;
    double e_tx = du - dvn * nx, e_ty = dv - dvn * ny, e_tz = dw - dvn * nz;
    double e_ap = dp + rho * c * dvn;
    double e_am = dp - rho * c * dvn;
    if (!(un > 0.0)) e_ent = e_tx = e_ty = e_tz = 0.0;
    if (!(un + c > 0.0)) e_ap = 0.0;
    if (!(un - c > 0.0)) e_am = 0.0;
    const double dp2 = 0.5 * (e_ap + e_am);
    const double dvn2 = (e_ap - e_am) / (2.0 * rho * c);
    const double drho2 = (dp2 - e_ent) / (c * c);
    put_prim(ph, U, N, n, ob[0] + drho2, ob[1] + e_tx + dvn2 * nx, ob[2] + e_ty + dvn2 * ny, ob[3] + e_tz + dvn2 * nz,
             ob[4] + dp2);
}

// Boundary nodes through the RK combination with L = 0 (U_out = a U^n +
// b U_in) before the boundary conditions of a stage, so that conditions that
// start from the boundary node's own value (non-reflecting faces) see the
// same value as in the update of interior nodes.  Face d of one launch skips
// nodes that also lie on a non-periodic face of a lower direction, so every
// node is combined once.
__global__ void k_bnd_rk(Geo g, double* Uout, const double* Uin, const double* Un, double a, double b, int d)
{
    const long long N = g.N;
    const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    const int ax = (d + 1) % 3, bx = (d + 2) % 3;
    const int dims[3] = {g.nx, g.ny, g.nz};
    const int na = dims[ax], nb = dims[bx];
    const long long nface = (long long)na * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * nface;
         e += (long long)gridDim.x * blockDim.x) {
        const int side = (int)(e / nface);
        const long long f = e % nface;
        int pos[3];
        pos[ax] = (int)(f % na);
        pos[bx] = (int)(f / na);
        pos[d] = side ? nd - 1 : 0;
        if (side && nd == 1) continue;
        bool owned = true;
        for (int q = 0; q < d; ++q)
            if (!g.per[q] && (pos[q] == 0 || pos[q] == dims[q] - 1)) owned = false;
        if (!owned) continue;
        const long long n = pos[0] + (long long)g.nx * (pos[1] + (long long)g.ny * pos[2]);
#pragma unroll
        for (int q = 0; q < 5; ++q) Uout[q * N + n] = mad(a, Un[q * N + n], b * Uin[q * N + n]);
    }
}

__global__ void k_bc(Geo g, Phys ph, BCData bc, double* U, int d, const double* tptr, const double* dtptr,
                     double tfrac)
{
    const long long N = g.N;
    const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    const long long s = d == 0 ? 1 : (d == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    const int dims[3] = {g.nx, g.ny, g.nz};
    const int na = dims[a], nb = dims[b];
    const long long nface = (long long)na * nb;
    const double t = (tptr ? *tptr : 0.0) + (dtptr ? tfrac * *dtptr : 0.0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * nface;
         e += (long long)gridDim.x * blockDim.x) {
        const int side = (int)(e / nface);
        const long long f = e % nface;
        const int type = side ? g.bc_hi[d] : g.bc_lo[d];
        if (type == 0 || type == 4) continue;  // periodic, or ghost layers filled by the halo exchange
        int pos[3];
        pos[a] = (int)(f % na);
        pos[b] = (int)(f / na);
        const int mb = side ? nd - 1 : 0, m1 = side ? nd - 2 : 1, m2 = side ? nd - 3 : 2;
        pos[d] = mb;
        const long long n = pos[0] + (long long)g.nx * (pos[1] + (long long)g.ny * pos[2]);
        const long long n1 = n + (long long)(m1 - mb) * s, n2 = n + (long long)(m2 - mb) * s;
        if (type == 3) {
            double o[5];
            cons_prim(ph, U, N, n1, o);
            put_prim(ph, U, N, n, o[0], o[1], o[2], o[3], o[4]);
        } else if (type == 5) {
            nonreflect_node(g, ph, U, n, n1, pos[0], pos[1], d, side ? 1.0 : -1.0);
        } else if (type == 2) {
            if (!bc.inflow) continue;
            const int jj = pos[1];
            const double* fl = bc.inflow;
            put_prim(ph, U, N, n, fl[jj], fl[g.ny + jj], fl[2 * g.ny + jj], fl[3 * g.ny + jj], fl[4 * g.ny + jj]);
        } else if (type == 1) {
            double o1[5], o2[5];
            cons_prim(ph, U, N, n1, o1);
            cons_prim(ph, U, N, n2, o2);
            const double pw = (4.0 * o1[4] - o2[4]) / 3.0;
            const double rhow = ph.gMa2 * pw / ph.Tw;
            double u = 0.0, v = 0.0, w = 0.0;
            if (d == 1 && side == 0 && bc.amp != 0.0 && bc.wall_x && bc.wall_z) {
                const double x = bc.wall_x[pos[0]], z = bc.wall_z[pos[2]];
                if (x >= bc.x0 && x <= bc.x1) {
                    const double pi = 3.14159265358979323846;
                    const double vn = bc.amp * sin(2.0 * pi * (x - bc.x0) / (bc.x1 - bc.x0)) *
                                      cos(2.0 * pi * bc.m * z / bc.Lz) * sin(bc.omega * t);
                    const long long mi = midx(g, pos[0], pos[1], n);
                    const double ex = metv(g, 3, mi), ey = metv(g, 4, mi), ez = metv(g, 5, mi);
                    const double nr = sqrt(ex * ex + ey * ey + ez * ez);
                    u = vn * ex / nr; v = vn * ey / nr; w = vn * ez / nr;
                }
            }
            put_prim(ph, U, N, n, rhow, u, v, w, pw);
        }
    }
}

// ---------------------------------------------------------------------------
// CFL time step (reading R16): max over nodes, as ordered bits of a non-
// negative double
// ---------------------------------------------------------------------------
template <class RT>
__global__ void k_cfl(Geo g, const RT* __restrict__ P, unsigned long long* out)
{
    const long long N = g.N;
    double mx = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        int i = (int)(n % g.nx);
        int j = (int)((n / g.nx) % g.ny);
        long long mi = midx(g, i, j, n);
        double u = P[N + n], v = P[2 * N + n], w = P[3 * N + n], c = P[6 * N + n];
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            double dx = metv(g, 3 * d, mi), dy = metv(g, 3 * d + 1, mi), dz = metv(g, 3 * d + 2, mi);
            s += fabs(dx * u + dy * v + dz * w) + c * sqrt(dx * dx + dy * dy + dz * dz);
        }
        mx = fmax(mx, s);
    }
    for (int off = 16; off; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// FMA-throughput probe: 8 independent dependency chains per thread
template <class T>
__global__ void k_fma_probe(T* out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = (T)(threadIdx.x + r) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) x[r] = x[r] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) s += x[r];
    if (s == (T)12345.678) out[0] = s;  // keeps the chains alive
}

// Self-check of the integer-pipe format conversions against the hardware
// cvt: f2d_exact over every float bit pattern; d2f_rn_int over 2^32 doubles
// drawn by SplitMix64 (Steele, Lea, Flood 2014) from their index, with
// exponents swept across and around float's range and the 29 cut-off
// fraction bits forced to the rounding edges (0, just below, at and just
// above one half, all ones) in five of every eight.  out: [0] floats
// checked, [1] float->double mismatches, [2] doubles with ok set, [3] their
// mismatches, [4] doubles whose ok flag disagrees with the stated range.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_check_conversions(unsigned long long* out)
{
    unsigned long long c[5] = {0, 0, 0, 0, 0};
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const double lo_ok = __longlong_as_double(0x3810000000000000ll);  // 2^-126
    const double hi_ok = __longlong_as_double(0x47f0000000000000ll);  // 2^128
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < (1ull << 32);
         v += stride) {
        const float f = __uint_as_float((unsigned)v);
        const double hw = (double)f, sw = f2d_exact(f);
        c[0] += 1;
        if (hw != hw ? sw == sw : __double_as_longlong(hw) != __double_as_longlong(sw)) c[1] += 1;

        const unsigned long long h = splitmix64(v), r = splitmix64(v ^ 0x5851f42d4c957f2dull);
        const unsigned sel = (unsigned)(h >> 55);
        // exponent fields 893 .. 1152 (float's range and two beyond each end) or
        // one of: zero/subnormal, smallest normal, largest finite, inf/NaN, 1.0,
        // and three far outside float's range
        const unsigned spec[8] = {0u, 1u, 2046u, 2047u, 1023u, 960u, 700u, 1300u};
        const unsigned long long ex = sel < 260u ? 893u + sel : spec[sel & 7u];
        unsigned long long fr = r & 0xfffffffffffffull;
        const unsigned long long edge[5] = {0ull, 0x0fffffffull, 0x10000000ull, 0x10000001ull, 0x1fffffffull};
        if ((v & 7u) < 5u) fr = (fr & ~0x1fffffffull) | edge[v & 7u];
        const double x = __longlong_as_double((long long)(((h & 1ull) << 63) | (ex << 52) | fr));
        bool ok;
        const float s = d2f_rn_int(x, ok);
        const bool want = x == 0.0 || (fabs(x) >= lo_ok && fabs(x) < hi_ok);
        if (ok != want) c[4] += 1;
        if (ok) {
            c[2] += 1;
            if (__float_as_uint(s) != __float_as_uint((float)x)) c[3] += 1;
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        unsigned long long t = c[q];
        for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(out + q, t);
    }
}

__global__ void k_set_scalar(double* dst, double v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

__global__ void k_advance_time(double* t, const double* dt)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t += *dt;
}

// ---------------------------------------------------------------------------
// kernels: single-block launches (grid = the block's tiles) ...
// ---------------------------------------------------------------------------
template <class RT>
__global__ void k_prim(SweepArgs A) { prim_body<RT>(A, blockIdx); }
__global__ void k_prim_mixed(SweepArgs A) { prim_mixed_body<false>(A, blockIdx); }
__global__ void k_sensor(SweepArgs A) { sensor_body<false>(A, blockIdx); }
__global__ void k_sensor32(SweepArgs A) { sensor32_body<false>(A, blockIdx); }
template <class R, int YB = 0, bool P8 = false, bool SENS = false>
__global__ void __launch_bounds__(256) k_visc_flux(SweepArgs A) { visc_node_body<R, YB, P8, SENS>(A, blockIdx); }
template <class R, int TZ>
__global__ void __launch_bounds__(256) k_visc_flux25(SweepArgs A) { visc25_body<R, TZ>(A, blockIdx); }
template <class R, int BX, int EP, bool CHAR = false, bool P8 = false>
__global__ void __launch_bounds__(BX) k_sweep_x(SweepArgs A) { sweep_x_body<R, BX, EP, CHAR, P8>(A, blockIdx); }
template <class R, int DIR, int EP, int TL, bool CHAR = false, bool P8 = false>
__global__ void __launch_bounds__(256, CHAR ? 1 : (sizeof(R) == 4 ? (TL == 16 ? 4 : 3) : 1)) k_sweep_t(SweepArgs A)
{
    sweep_t_body<R, DIR, EP, TL, CHAR, P8>(A, blockIdx);
}
template <class R, int EP>
__global__ void __launch_bounds__(XW) k_sweep_xw(SweepArgs A, int seg_len) { sweep_xw_body<R, EP>(A, blockIdx, seg_len); }
template <class R, int DIR, int EP>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_sweep_w(SweepArgs A) { sweep_w_body<R, DIR, EP>(A, blockIdx); }
template <int DIR, int EP>
__global__ void __launch_bounds__(256, 2) k_sweep_wt(SweepArgs A, const __grid_constant__ TmaRowMaps maps)
{
    sweep_wt_body<DIR, EP>(A, maps, blockIdx);
}

// ---------------------------------------------------------------------------
// ... and persistent batched launches over an ensemble of uneven blocks: one
// launch per kernel kind covers the tiles of every block; CTAs walk a work
// list (item -> block by binary search over the per-block tile prefix sums,
// then the block-local tile coordinates) with a grid-size stride.
// ---------------------------------------------------------------------------
static_assert(sizeof(SweepArgs) % sizeof(int) == 0, "argument record copied as words");

struct BatchMap {
    const SweepArgs* tbl;  // [nb] per-block arguments of this stage
    const int* prefix;     // [nb+1] tile prefix sums for this kernel kind
    const int* gdim;       // [nb][3] per-block tile grid of this kernel kind
    int nb;
};

__device__ __forceinline__ int batch_find(const BatchMap& m, int item, uint3* v)
{
    int lo = 0, hi = m.nb;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(m.prefix + mid) <= item) lo = mid;
        else hi = mid;
    }
    const int local = item - __ldg(m.prefix + lo);
    const int gx = __ldg(m.gdim + 3 * lo), gy = __ldg(m.gdim + 3 * lo + 1);
    v->x = local % gx;
    v->y = (local / gx) % gy;
    v->z = local / (gx * gy);
    return lo;
}

// the item range [lo, hi) and tile grid (gx, gy) of the block a CTA worked
// on last: the next item usually lies in the same block, and then needs no
// search over the prefix sums
struct BatchRange {
    int lo, hi, gx, gy;
};

__device__ __forceinline__ int batch_find_cached(const BatchMap& m, int item, uint3* v, int cached, BatchRange& r)
{
    if (cached < 0 || item < r.lo || item >= r.hi) {
        cached = batch_find(m, item, v);
        r.lo = __ldg(m.prefix + cached);
        r.hi = __ldg(m.prefix + cached + 1);
        r.gx = __ldg(m.gdim + 3 * cached);
        r.gy = __ldg(m.gdim + 3 * cached + 1);
        return cached;
    }
    const int local = item - r.lo;
    v->x = local % r.gx;
    v->y = (local / r.gx) % r.gy;
    v->z = local / (r.gx * r.gy);
    return cached;
}

// CONTIG: each CTA takes a contiguous range of items (node kernels: its
// items stay in one block); otherwise items are dealt round-robin, so CTAs
// that run at the same time work on neighbouring tiles and share their halos
// in L2.  The block's argument record is copied to shared memory when a CTA
// moves to a new block, so the bodies read it from shared memory.
#define BATCH_LOOP(BODY, SYNC, CONTIG)                                                                \
    __shared__ __align__(16) SweepArgs sA;                                                            \
    constexpr int AW = (int)(sizeof(SweepArgs) / sizeof(int));                                        \
    int cached = -1;                                                                                  \
    BatchRange rng{0, 0, 1, 1};                                                                       \
    const int total = __ldg(m.prefix + m.nb);                                                         \
    const int per_cta = CONTIG ? (total + gridDim.x - 1) / gridDim.x : 1;                             \
    const int item_end = CONTIG ? min(total, ((int)blockIdx.x + 1) * per_cta) : total;                \
    const int item_step = CONTIG ? 1 : (int)gridDim.x;                                                \
    for (int item = blockIdx.x * per_cta; item < item_end; item += item_step) {                       \
        uint3 v;                                                                                      \
        const int b = batch_find_cached(m, item, &v, cached, rng);                                    \
        if (b != cached) {                                                                            \
            __syncthreads();                                                                          \
            const int* src = reinterpret_cast<const int*>(m.tbl + b);                                 \
            for (int w = threadIdx.x; w < AW; w += blockDim.x) reinterpret_cast<int*>(&sA)[w] = src[w];\
            __syncthreads();                                                                          \
            cached = b;                                                                               \
        }                                                                                             \
        BODY(sA, v);                                                                                  \
        if (SYNC) __syncthreads();                                                                    \
    }

template <class RT>
__global__ void kb_prim(BatchMap m) { BATCH_LOOP((prim_body<RT, true>), false, true) }
__global__ void kb_prim_mixed(BatchMap m) { BATCH_LOOP(prim_mixed_body<true>, false, true) }
__global__ void kb_sensor(BatchMap m) { BATCH_LOOP(sensor_body<true>, false, true) }
__global__ void kb_sensor32(BatchMap m) { BATCH_LOOP(sensor32_body<true>, false, true) }
// the learned sensor over an ensemble: items are (column x, column y, zeta
// segment of tz planes) of every block; the weights are staged once per CTA
template <class RT>
__global__ void __launch_bounds__(256, 2) kb_sensor_mlp(BatchMap m, MlpArgs W, int tz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpWalkSmem& S = *reinterpret_cast<MlpWalkSmem*>(smem_raw);
    mlp_stage_weights(S.w, W);
    uint32_t phase = 0;
    auto body = [&](const SweepArgs& A, uint3 v) { sensor_mlp_col<RT>(A, W, S, v, tz, phase); };
    BATCH_LOOP(body, true, false)
}
template <class RT>
__global__ void __launch_bounds__(256, 3) kb_sensor_mlp_tc(BatchMap m, MlpArgs W, int tz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpTcSmem& S = *reinterpret_cast<MlpTcSmem*>(smem_raw);
    mlp_tc_setup(S, W);
    uint32_t phase = 0;
    auto body = [&](const SweepArgs& A, uint3 v) { sensor_mlp_col<RT>(A, W, S, v, tz, phase); };
    BATCH_LOOP(body, true, false)
    mlp_tc_teardown(S);
}
template <class R, int TZ>
__global__ void __launch_bounds__(256) kb_visc_flux25(BatchMap m) { BATCH_LOOP((visc25_body<R, TZ>), true, false) }
// P8: every block periodic in every direction with 8th-order viscous terms
// (the instantiations without order and closure decisions, as for one block)
// SENS (FP32): the tiles also write the plain sensor's classes
template <class R, bool P8 = false, bool SENS = false>
__global__ void __launch_bounds__(128) kb_visc_flux_tiles(BatchMap m)
{
    BATCH_LOOP((visc_node_body<R, 4, P8, SENS>), false, false)
}
template <class R, int BX, int EP, bool P8 = false>
__global__ void __launch_bounds__(BX) kb_sweep_x(BatchMap m)
{
    BATCH_LOOP((sweep_x_body<R, BX, EP, false, P8>), true, false)
}
// walking xi sweep over whole lines (items: one x-line of one block)
template <class R, int EP>
__device__ __forceinline__ void sweep_xw_line(const SweepArgs& A, uint3 vb) { sweep_xw_body<R, EP>(A, vb, 1 << 30); }
template <class R, int EP>
__global__ void __launch_bounds__(XW) kb_sweep_xw(BatchMap m) { BATCH_LOOP((sweep_xw_line<R, EP>), true, false) }
template <class R, int DIR, int EP, int TL, bool P8 = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? (TL == 16 ? 4 : 3) : 1) kb_sweep_t(BatchMap m)
{
    BATCH_LOOP((sweep_t_body<R, DIR, EP, TL, false, P8>), true, false)
}
template <class R, int DIR, int EP, bool P8 = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) kb_sweep_w(BatchMap m)
{
    BATCH_LOOP((sweep_w_body<R, DIR, EP, P8>), true, false)
}

}  // namespace cfdk
