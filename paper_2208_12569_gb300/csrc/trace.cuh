// Persistent field-line tracer (templated on the traced precision T).
//
// Method (Zhang et al. 2022):
//   - field-line equation dr/ds = B/|B| (Sec. 2.1, Eq. rb), integrated in index
//     coordinates xi = (r - o)/d with d xi/d tau = bt/|bt|, bt_a = B_a/d_a, so
//     tau, step and tol are in cells (Sec. 2.3); physical length dl/dtau =
//     |B|/|bt| and the twist integrand (curl B . B)/(4 pi B^2) dl/dtau (Eq. tw)
//     ride along as two extra components;
//   - B and curl B between nodes by trilinear interpolation with a floor cell
//     lookup clamped to [0, n-2] (Sec. 2.2, Eqs. interp, w0, w1);
//   - Fehlberg's RKF45 pair with the 4th-order solution propagated; a trial is
//     accepted when the position error (cells) is <= the line's tolerance;
//     with q = (tol/err)^(1/4) taken as two correctly rounded square roots,
//     growth min(4, 0.9 q), shrink max(0.1, 0.9 q), h in [h_min, h_max], a
//     reject at h_min is accepted and flagged (Sec. 2.3);
//   - at the box exit the accepted step is discarded and one RKF45 step is
//     taken from the previous point with the face-normal index coordinate as
//     the independent variable, landing exactly on the face (the paper's "move
//     one step back", Sec. 2.1); grazing exits halve h and retry;
//   - per-line tolerance tol_perp max(|Bn0/B|, rot_thresh)^1.5 (Sec. 4, Eq.
//     tol); seeds of an interior S0 below rot_thresh are queued for the rotated
//     S0 and traced with tol_perp.
//
// GPU design: one lane per line; a warp takes tiles of 8x4 neighbouring seeds
// from a device work counter (persistent grid) so that the 32 lines of a warp
// gather from the same cells; a lane whose line is done takes the next seed
// before the next trial step. Normal trials and exit steps share one 6-stage
// code path, so a warp only diverges at line start and end. The state is
// stepped in T; the error norm, the tolerance and the Tw/length sums are FP64.
// The FP64 instantiation is built without floating-point contraction and
// evaluates every expression in the order of its definition (Eq. interp term
// by term, the 4th- and 5th-order solutions formed separately), because the
// adaptive step sequence amplifies any rounding difference by orders of
// magnitude per step: that way it reproduces a plain evaluation of the method
// to the last bit. The FP32 instantiation uses the fast forms.
#pragma once

#include <math.h>

#include "fqsl_internal.cuh"

// Resident 128-thread blocks per SM asked of the FP64 RKF45 tracers (not the
// Method II or fixed-step ones): their latency (FP64 divisions and square
// roots on GB300's narrow FP64 pipe) wants warps more than registers. 8 blocks
// (64 registers, the rest spilled to L1) measured fastest: 92.5 ms per
// 1024x1024 map of the 256x256x128 monopole cube against 108.9 ms at 168
// registers and 3 blocks. The fixed-step FP64 map measured slower with it
// (8.5 against 8.9 M Q+Tw/s) and keeps its registers.
#ifndef FQSL_TRACE_F64_MINB
#define FQSL_TRACE_F64_MINB 8
#endif

namespace fqsl {
namespace trace {

constexpr int kChunk = kTileU * kTileV;  // work items per queue grab

// Fehlberg 4(5) coefficients.
template <typename T>
struct Fehlberg {
    static __device__ __forceinline__ T a(int s, int r)
    {
        // lower-triangular stage matrix, row s (1..5), column r < s
        const double A[6][5] = {{0, 0, 0, 0, 0},
                                {1.0 / 4.0, 0, 0, 0, 0},
                                {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
                                {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
                                {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
                                {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
        return (T)A[s][r];
    }
    static __device__ __forceinline__ T b4(int s)
    {
        const double B[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
        return (T)B[s];
    }
    static __device__ __forceinline__ T b5(int s)
    {
        const double B[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
        return (T)B[s];
    }
    // 5th minus 4th order weights (error estimate)
    static __device__ __forceinline__ T e(int s)
    {
        const double E[6] = {16.0 / 135.0 - 25.0 / 216.0,
                             0.0,
                             6656.0 / 12825.0 - 1408.0 / 2565.0,
                             28561.0 / 56430.0 - 2197.0 / 4104.0,
                             -9.0 / 50.0 + 1.0 / 5.0,
                             2.0 / 55.0};
        return (T)E[s];
    }
};

// Kutta's 3/8 rule (fixed-step scheme, Sec. 2.3).
template <typename T>
struct Kutta38 {
    static __device__ __forceinline__ T a(int s, int r)
    {
        const double A[4][3] = {{0, 0, 0}, {1.0 / 3.0, 0, 0}, {-1.0 / 3.0, 1.0, 0}, {1.0, -1.0, 1.0}};
        return (T)A[s][r];
    }
    static __device__ __forceinline__ T b(int s)
    {
        const double B[4] = {1.0 / 8.0, 3.0 / 8.0, 3.0 / 8.0, 1.0 / 8.0};
        return (T)B[s];
    }
};

// The stages of a trial: SCH 0 = RKF45 (6 stages, 4th-order solution and the
// 5th-order error estimate), 1 = the 3/8 rule (4 stages, no estimate).
template <typename T, int SCH>
struct Tab {
    static constexpr int N = SCH ? 4 : 6;
    static __device__ __forceinline__ T a(int s, int r) { return SCH ? Kutta38<T>::a(s, r) : Fehlberg<T>::a(s, r); }
    static __device__ __forceinline__ T b(int s) { return SCH ? Kutta38<T>::b(s) : Fehlberg<T>::b4(s); }
};

// ---------------------------------------------------------------------------
// trilinear gather of B and curl B at index position (x, y, z)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_node(const FieldView &f, long long node, float &bx, float &by, float &bz,
                                          float &jx, float &jy, float &jz)
{
    const float4 *r = (const float4 *)f.rec + 2 * node;
    const float4 a = __ldg(r);
    const float4 b = __ldg(r + 1);
    bx = a.x;
    by = a.y;
    bz = a.z;
    jx = a.w;
    jy = b.x;
    jz = b.y;
}

__device__ __forceinline__ void load_node(const FieldView &f, long long node, double &bx, double &by, double &bz,
                                          double &jx, double &jy, double &jz)
{
    const double2 *r = (const double2 *)f.rec + 4 * node;
    const double2 a = __ldg(r);
    const double2 b = __ldg(r + 1);
    const double2 c = __ldg(r + 2);
    bx = a.x;
    by = a.y;
    bz = b.x;
    jx = b.y;
    jy = c.x;
    jz = c.y;
}


// FP64 cells on the integer pipe (GB300's FP64 pipe is the FP64 tracer's
// bound, and it would also run the floor, clamps and conversions): the cell
// min(max(floor(x), 0), n - 2) as an integer (NaN and x < 0 give 0,
// x >= n - 2 and +inf give n - 2), read off the double's exponent and mantissa.
__device__ __forceinline__ int cell_floor64(double x, int n)
{
    const long long u = __double_as_longlong(x);
    const int top = n - 2;
    if (u < 0) return 0;  // sign set: negative, -0, a negative NaN
    const int e = (int)(u >> 52);
    if (e == 0x7ff) return (u & 0xfffffffffffffLL) ? 0 : top;  // NaN, +inf
    if (e < 1023) return 0;                                    // [0, 1)
    if (e >= 1023 + 31) return top;
    const unsigned long long m = ((unsigned long long)u & 0xfffffffffffffULL) | (1ULL << 52);
    const long long c = (long long)(m >> (52 - (e - 1023)));
    return c > top ? top : (int)c;
}

// float -> double, exactly, on the integer pipe (GB300's narrow FP64 pipe
// would also run the hardware conversion). Normal
// numbers move their exponent from bias 127 to 1023 and their mantissa to the
// top of the double's; subnormals are normalised by their leading one; zeros,
// infinities and NaNs keep their class.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned m = b & 0x7fffffu;
    unsigned hi, lo;
    if (e == 0xffu) {
        hi = sign | 0x7ff00000u | (m >> 3);
        lo = m << 29;
    } else if (e != 0u) {
        hi = sign | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    } else if (m == 0u) {
        hi = sign;
        lo = 0u;
    } else {
        // m 2^-149 with its leading one at bit p: 1.f 2^(p - 149)
        const int p = 31 - __clz(m);
        const unsigned mm = (m << (23 - p)) & 0x7fffffu;
        hi = sign | ((unsigned)(p + 874) << 20) | (mm >> 3);
        lo = mm << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// an integer in [0, 2^31) as the double of the same value (exact)
__device__ __forceinline__ double int_f64(int c)
{
    if (c <= 0) return 0.0;
    const int p = 31 - __clz(c);
    const unsigned long long m = ((unsigned long long)c << (52 - p)) & 0xfffffffffffffULL;
    return __longlong_as_double((long long)(((unsigned long long)(p + 1023) << 52) | m));
}

// i + 1/2 as a double (exact): (2i + 1) made a double by its bits, halved
// by its exponent
__device__ __forceinline__ double half_odd(unsigned i)
{
    if (i >= (1u << 30)) return (double)i + 0.5;
    const double d = int_f64((int)(2u * i + 1u));
    return __longlong_as_double(__double_as_longlong(d) - (1LL << 52));
}

// One 32-byte FP32 node record in a single 256-bit read-only load (records are
// 32-byte aligned: the allocation is, and every record offset is a multiple of
// 32). Returns Bx, By, Bz, Jx, Jy, Jz.
#pragma nv_diag_suppress 550  // the two padding floats of the record are loaded and dropped
__device__ __forceinline__ void load_rec32(const char *p, float &b0, float &b1, float &b2, float &j0, float &j1,
                                           float &j2)
{
    float pad0, pad1;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(b0), "=f"(b1), "=f"(b2), "=f"(j0), "=f"(j1), "=f"(j2), "=f"(pad0), "=f"(pad1)
        : "l"(p));
}
#pragma nv_diag_default 550

// The B half of a record (its first 16 bytes) in one 128-bit load, for
// evaluations whose curl B is not used.
#pragma nv_diag_suppress 550
__device__ __forceinline__ void load_rec32_b(const char *p, float &b0, float &b1, float &b2)
{
    float j0;
    asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(b0), "=f"(b1), "=f"(b2), "=f"(j0) : "l"(p));
}
#pragma nv_diag_default 550

// Exact integer value of a float that holds an integer in [0, 2^23): adding
// 2^23 puts it in the low mantissa bits. (A float -> 64-bit integer conversion
// runs on GB300's narrow FP64 pipe; this is one FADD and one integer op.)
__device__ __forceinline__ int small_int(float c) { return __float_as_int(c + 8388608.f) - 0x4B000000; }

// FP32: weights as products of per-axis weights, corners grouped by (y, z);
// 32-bit cell arithmetic and byte strides (field_create keeps every axis below
// 2^23 nodes and the cube below 2^31 nodes; sz32 = 0 marks a z stride that
// does not fit 32 bits).
// The 8 corners of cell node (its lowest corner) with per-axis weights w (the
// upper node's) and u = 1 - w. wj = false: B only (J = 0), half the bytes.
__device__ __forceinline__ void gather_cell32(const FieldView &f, unsigned node, float wx, float wy, float wz,
                                              float ux, float uy, float uz, float B[3], float J[3], bool wj = true)
{
    const char *p00 = (const char *)f.rec + (size_t)node * 32u;
    const size_t szb = f.sz32 ? (size_t)f.sz32 : (size_t)f.nx * (size_t)f.ny * 32u;
    const char *pc[4] = {p00, p00 + f.sy32, p00 + szb, p00 + szb + f.sy32};
    const float wyz[4] = {uy * uz, wy * uz, uy * wz, wy * wz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        B[c] = 0.f;
        J[c] = 0.f;
    }
#pragma unroll
    for (int qp = 0; qp < 4; qp++) {
#pragma unroll
        for (int m = 0; m < 2; m++) {
            float r0, r1, r2, r3 = 0.f, r4 = 0.f, r5 = 0.f;
            if (wj) load_rec32(pc[qp] + 32 * m, r0, r1, r2, r3, r4, r5);
            else load_rec32_b(pc[qp] + 32 * m, r0, r1, r2);
            const float w = (m ? wx : ux) * wyz[qp];
            B[0] += w * r0;
            B[1] += w * r1;
            B[2] += w * r2;
            if (wj) {
                J[0] += w * r3;
                J[1] += w * r4;
                J[2] += w * r5;
            }
        }
    }
}

__device__ __forceinline__ void gather(const FieldView &f, float x, float y, float z, float B[3], float J[3],
                                       bool wj = true)
{
    const float cx = fminf(fmaxf(floorf(x), 0.f), f.cmax[0]);
    const float cy = fminf(fmaxf(floorf(y), 0.f), f.cmax[1]);
    const float cz = fminf(fmaxf(floorf(z), 0.f), f.cmax[2]);
    const float wx = x - cx, wy = y - cy, wz = z - cz;
    const float ux = 1.f - wx, uy = 1.f - wy, uz = 1.f - wz;
    const unsigned node = ((unsigned)small_int(cz) * (unsigned)f.ny + (unsigned)small_int(cy)) * (unsigned)f.nx +
                          (unsigned)small_int(cx);
    gather_cell32(f, node, wx, wy, wz, ux, uy, uz, B, J, wj);
}

// FP64: Eq. interp term by term, omega_0 = (i+1) - xi and omega_1 = 1 - omega_0
// (Eqs. w0, w1 in cells), summed over m (x), n (y), p (z) in that nesting.
// Built without contraction, this is the plain evaluation of the definition.
// (wj: accepted for the common interface; the FP64 gather always forms J)
__device__ __forceinline__ void gather(const FieldView &f, double x, double y, double z, double B[3], double J[3],
                                       bool wj = true)
{
    // (c + 1 as a double is exact, so int_f64(c + 1) is the c + 1.0 of the form)
    const int c[3] = {cell_floor64(x, f.nx), cell_floor64(y, f.ny), cell_floor64(z, f.nz)};
    const double xi[3] = {x, y, z};
    double w[3][2];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        w[a][0] = int_f64(c[a] + 1) - xi[a];
        w[a][1] = 1.0 - w[a][0];
    }
    const long long sy = f.nx, sz = (long long)f.nx * f.ny;
    const long long base = (long long)c[2] * sz + (long long)c[1] * sy + (long long)c[0];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        B[k] = 0.0;
        J[k] = 0.0;
    }
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const double wt = w[0][m] * w[1][q] * w[2][p];
                double bx, by, bz, jx, jy, jz;
                load_node(f, base + p * sz + q * sy + m, bx, by, bz, jx, jy, jz);
                B[0] += wt * bx;
                B[1] += wt * by;
                B[2] += wt * bz;
                J[0] += wt * jx;
                J[1] += wt * jy;
                J[2] += wt * jz;
            }
}

// ---------------------------------------------------------------------------
// Stretched (rectilinear) grids (Sec. 2.2): the cell of a coordinate is the
// largest i in [0, n-2] with x_i <= x (below x_0, and NaN: cell 0). The paper
// finds it by binary search. Here the coordinate's bucket names a cell and the
// next node, one comparison picks the cell, and its record (both nodes) checks
// it; a bucket index that rounding moved to a neighbour fails the check and is
// walked to the right cell (each walk moves one way and stops at the axis
// ends), so every x gets the binary search's cell.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int axis_n(const FieldView &f, int a) { return a == 0 ? f.nx : (a == 1 ? f.ny : f.nz); }

// The walk of a bucket index that rounding moved into a neighbouring bucket
// (rare; kept out of line to keep the tracer's code small).
static __device__ __noinline__ int rect_walk32(const float4 *__restrict__ cells, int n, float x, int c)
{
    if (!(x >= 0.f)) return 0;
    while (c < n - 2 && x >= __ldg(cells + c).y) c++;
    while (c > 0 && x < __ldg(cells + c).x) c--;
    return c;
}

// FP32: cell of x (relative to x_0) with its record {x_c, x_{c+1}, 1/width}.
// One 32-byte load of the bucket holds both cells a point of the bucket can
// fall in.
__device__ __forceinline__ int rect_cell(const FieldView &f, int a, float x, float4 &cr)
{
    const int n = axis_n(f, a);
    const float bf = fminf(fmaxf(x, 0.f) * f.bsc32[a], (float)(f.nbkt[a] - 1));  // NaN -> bucket 0
    float c0, x0, x1, r0, thr, x2, r1, pad;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(c0), "=f"(x0), "=f"(x1), "=f"(r0), "=f"(thr), "=f"(x2), "=f"(r1), "=f"(pad)
        : "l"(f.bk32[a] + 2 * small_int(floorf(bf))));
    int c = __float_as_int(c0);
    if (x >= thr) {
        c++;
        cr = make_float4(x1, x2, r1, 0.f);
    } else {
        cr = make_float4(x0, x1, r0, 0.f);
    }
    if ((c > 0 && !(x >= cr.x)) || (c < n - 2 && x >= cr.y)) {
        // the bucket index was rounded into a neighbour (or x is NaN)
        c = rect_walk32(f.cell32[a], n, x, c);
        cr = __ldg(f.cell32[a] + c);
    }
    return c;
}

// FP64: cell of x (physical) with its nodes {x_c, x_{c+1}}
__device__ __forceinline__ int rect_cell(const FieldView &f, int a, double x, double2 &cr)
{
    const int n = axis_n(f, a);
    int c = 0;
    if (x >= f.lo64[a]) {
        const double bf = (x - f.lo64[a]) * f.bsc64[a];
        c = __ldg(f.bkt[a] + (bf < (double)(f.nbkt[a] - 1) ? (int)bf : f.nbkt[a] - 1));
    }
    cr = __ldg(f.cell64[a] + c);
    while (c < n - 2 && x >= cr.y) cr = __ldg(f.cell64[a] + (++c));
    while (c > 0 && x < cr.x) cr = __ldg(f.cell64[a] + (--c));
    return c;
}

// The cells of a point on the three axes with their records.
template <typename T>
struct RectCells;
template <>
struct RectCells<float> {
    int c[3];
    float4 r[3];
};
template <>
struct RectCells<double> {
    int c[3];
    double2 r[3];
};

template <typename T>
__device__ __forceinline__ void rect_cells(const FieldView &f, T x, T y, T z, RectCells<T> &rc)
{
    rc.c[0] = rect_cell(f, 0, x, rc.r[0]);
    rc.c[1] = rect_cell(f, 1, y, rc.r[1]);
    rc.c[2] = rect_cell(f, 2, z, rc.r[2]);
}

// FP32 on a stretched grid: state coordinates relative to the first node,
// omega_0 = (x_{i+1} - x) / (x_{i+1} - x_i) with the reciprocal width (Eq. w0)
__device__ __forceinline__ void gather_rect_at(const FieldView &f, float x, float y, float z, const RectCells<float> &rc,
                                               float B[3], float J[3], bool wj = true)
{
    const float ux = (rc.r[0].y - x) * rc.r[0].z, uy = (rc.r[1].y - y) * rc.r[1].z, uz = (rc.r[2].y - z) * rc.r[2].z;
    const unsigned node =
        ((unsigned)rc.c[2] * (unsigned)f.ny + (unsigned)rc.c[1]) * (unsigned)f.nx + (unsigned)rc.c[0];
    gather_cell32(f, node, 1.f - ux, 1.f - uy, 1.f - uz, ux, uy, uz, B, J, wj);
}

// FP64 on a stretched grid: Eqs. interp, w0, w1 as written in physical
// coordinates, the sum nested as in the uniform FP64 gather
__device__ __forceinline__ void gather_rect_at(const FieldView &f, double x, double y, double z,
                                               const RectCells<double> &rc, double B[3], double J[3], bool wj = true)
{
    const double xi[3] = {x, y, z};
    long long c[3];
    double w[3][2];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double2 cr = rc.r[a];
        c[a] = rc.c[a];
        w[a][0] = (cr.y - xi[a]) / (cr.y - cr.x);
        w[a][1] = 1.0 - w[a][0];
    }
    const long long sy = f.nx, sz = (long long)f.nx * f.ny;
    const long long base = c[2] * sz + c[1] * sy + c[0];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        B[k] = 0.0;
        J[k] = 0.0;
    }
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const double wt = w[0][m] * w[1][q] * w[2][p];
                double bx, by, bz, jx, jy, jz;
                load_node(f, base + p * sz + q * sy + m, bx, by, bz, jx, jy, jz);
                B[0] += wt * bx;
                B[1] += wt * by;
                B[2] += wt * bz;
                J[0] += wt * jx;
                J[1] += wt * jy;
                J[2] += wt * jz;
            }
}

template <typename T>
__device__ __forceinline__ void gather_rect(const FieldView &f, T x, T y, T z, T B[3], T J[3], bool wj = true)
{
    RectCells<T> rc;
    rect_cells(f, x, y, z, rc);
    gather_rect_at(f, x, y, z, rc, B, J, wj);
}

// wj = false: B only where the precision allows (FP32 loads half of each record)
template <bool RECT, typename T>
__device__ __forceinline__ void gatherg(const FieldView &f, T x, T y, T z, T B[3], T J[3], bool wj = true)
{
    if constexpr (RECT) gather_rect(f, x, y, z, B, J, wj);
    else gather(f, x, y, z, B, J, wj);
}

// Box bounds in state coordinates: [0, n-1] cells; on a stretched grid the
// first and last node (FP64: physical; FP32: relative to the first node).
template <typename T, bool RECT>
__device__ __forceinline__ T lo_of(const FieldView &f, int a)
{
    if constexpr (RECT && sizeof(T) == 8) return (T)f.lo64[a];
    else return (T)0;
}

template <typename T, bool RECT>
__device__ __forceinline__ T hi_of(const FieldView &f, int a)
{
    if constexpr (RECT) {
        if constexpr (sizeof(T) == 8) return (T)f.hi64[a];
        else return (T)f.hi32[a];
    } else {
        return (T)(axis_n(f, a) - 1);
    }
}

// FP64: the cells' widths; FP32: their reciprocals
__device__ __forceinline__ void dd_of(const RectCells<double> &rc, double dd[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) dd[a] = rc.r[a].y - rc.r[a].x;
}
__device__ __forceinline__ void dd_of(const RectCells<float> &rc, float dd[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) dd[a] = rc.r[a].z;
}

// The step's scale per axis, fixed at the start of a trial: FP64 the width
// of the cell holding the start point (the spacing on a uniform grid), FP32
// its reciprocal (Sec. 2.3: step and tol scaled per cell).
template <typename T, bool RECT>
__device__ __forceinline__ void step_dd(const FieldView &f, T x, T y, T z, T dd[3])
{
    if constexpr (!RECT) {
#pragma unroll
        for (int a = 0; a < 3; a++) dd[a] = sizeof(T) == 8 ? (T)f.d[a] : (T)f.rd[a];
    } else {
        RectCells<T> rc;
        rect_cells(f, x, y, z, rc);
        dd_of(rc, dd);
    }
}

// state <-> physical coordinates (double): (r - o)/d and o + d x on a uniform
// grid (and for FP32 on a stretched one, where o is the first node and d = 1);
// the FP64 state on a stretched grid is the physical position.
template <typename T, bool RECT>
__device__ __forceinline__ double state_of(const FieldView &f, double r, int a)
{
    if constexpr (RECT && sizeof(T) == 8) return r;
    else return (r - f.o[a]) / f.d[a];
}

// Right-hand side in index space: out = {F (3), dl/dtau, dTw/dtau}.
// Returns false on a null / non-finite field. wj = false (a stage whose Tw
// weight is zero): dTw/dtau = 0 without loading curl B.
__device__ __forceinline__ bool rhs(const FieldView &f, const float invd[3], float sgn, float x, float y, float z,
                                    float out[5], bool wj = true)
{
    float B[3], J[3];
    gather(f, x, y, z, B, J, wj);
    const float b0 = B[0] * invd[0], b1 = B[1] * invd[1], b2 = B[2] * invd[2];
    const float bb = b0 * b0 + b1 * b1 + b2 * b2;
    const float BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    if (!(bb > 0.f) || !(bb < INFINITY)) return false;
    const float inv = rsqrtf(bb);
    const float s = sgn * inv;
    out[0] = b0 * s;
    out[1] = b1 * s;
    out[2] = b2 * s;
    const float dl = sqrtf(BB) * inv;
    out[3] = dl;
    const float JB = J[0] * B[0] + J[1] * B[1] + J[2] * B[2];
    out[4] = wj ? __fdividef(JB * dl, 12.566370614359172f * BB) : 0.f;
    return true;
}

// FP64: bt_a = B_a / d_a, F = sigma bt / |bt|, dl/dtau = |B| / |bt|,
// dTw/dtau = (J.B) / (4 pi B^2) dl/dtau, each as written.
// (wj: accepted for the common interface; FP64 always forms dTw/dtau)
__device__ __forceinline__ bool rhs(const FieldView &f, const double d[3], double sgn, double x, double y,
                                    double z, double out[5], bool wj = true)
{
    double B[3], J[3];
    gather(f, x, y, z, B, J);
    // (on a unit-spacing grid B_a / 1 = B_a exactly: no division)
    const double bt[3] = {f.unit ? B[0] : B[0] / d[0], f.unit ? B[1] : B[1] / d[1], f.unit ? B[2] : B[2] / d[2]};
    const double bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
    const double BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    if (!(bb > 0.0) || !(bb < INFINITY)) return false;
    const double nbt = sqrt(bb), nB = sqrt(BB);
    out[0] = sgn * bt[0] / nbt;
    out[1] = sgn * bt[1] / nbt;
    out[2] = sgn * bt[2] / nbt;
    const double dl = nB / nbt;
    out[3] = dl;
    out[4] = (J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) / (12.566370614359172 * BB) * dl;
    return true;
}

// Stretched grid: bt_a = B_a / D_a with the step's cell widths D, and the
// physical velocity F = sigma B / |bt| (FP32: rw = 1/D).
__device__ __forceinline__ bool rhs_rect(const FieldView &f, const float rw[3], float sgn, float x, float y, float z,
                                         float out[5], const RectCells<float> *pre = nullptr, bool wj = true)
{
    float B[3], J[3];
    if (pre) gather_rect_at(f, x, y, z, *pre, B, J, wj);
    else gather_rect(f, x, y, z, B, J, wj);
    const float b0 = B[0] * rw[0], b1 = B[1] * rw[1], b2 = B[2] * rw[2];
    const float bb = b0 * b0 + b1 * b1 + b2 * b2;
    const float BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    if (!(bb > 0.f) || !(bb < INFINITY)) return false;
    const float inv = rsqrtf(bb);
    const float s = sgn * inv;
    out[0] = B[0] * s;
    out[1] = B[1] * s;
    out[2] = B[2] * s;
    const float dl = sqrtf(BB) * inv;
    out[3] = dl;
    const float JB = J[0] * B[0] + J[1] * B[1] + J[2] * B[2];
    out[4] = wj ? __fdividef(JB * dl, 12.566370614359172f * BB) : 0.f;
    return true;
}

__device__ __forceinline__ bool rhs_rect(const FieldView &f, const double D[3], double sgn, double x, double y,
                                         double z, double out[5], const RectCells<double> *pre = nullptr,
                                         bool wj = true)
{
    double B[3], J[3];
    if (pre) gather_rect_at(f, x, y, z, *pre, B, J);
    else gather_rect(f, x, y, z, B, J);
    const double bt[3] = {B[0] / D[0], B[1] / D[1], B[2] / D[2]};
    const double bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
    const double BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    if (!(bb > 0.0) || !(bb < INFINITY)) return false;
    const double nbt = sqrt(bb), nB = sqrt(BB);
    out[0] = sgn * B[0] / nbt;
    out[1] = sgn * B[1] / nbt;
    out[2] = sgn * B[2] / nbt;
    const double dl = nB / nbt;
    out[3] = dl;
    out[4] = (J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) / (12.566370614359172 * BB) * dl;
    return true;
}

// pre (stretched grid): the point's cells, already searched
template <bool RECT, typename T>
__device__ __forceinline__ bool rhsg(const FieldView &f, const T dd[3], T sgn, T x, T y, T z, T out[5],
                                     const RectCells<T> *pre = nullptr, bool wj = true)
{
    if constexpr (RECT) return rhs_rect(f, dd, sgn, x, y, z, out, pre, wj);
    else return rhs(f, dd, sgn, x, y, z, out, wj);
}

// ---------------------------------------------------------------------------
// Method II: grad(B/|B|) at a point (Sec. 4): way 1 interpolates the node grid
// of Eq. grad_B trilinearly, way 2 differences B/|B| at xi +- eps e_a.
// G[a][b] = d(B_b/|B|)/dx_a in physical units. Returns false on a null field.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gather_grad_cell(const FieldView &f, long long base, float wx, float wy, float wz,
                                                 float ux, float uy, float uz, float G[3][3])
{
    const long long sy = f.nx, sz = (long long)f.nx * f.ny;
    const float4 *g = (const float4 *)f.grad;
    const float wyz[4] = {uy * uz, wy * uz, uy * wz, wy * wz};
    float acc[9];
#pragma unroll
    for (int c = 0; c < 9; c++) acc[c] = 0.f;
#pragma unroll
    for (int qp = 0; qp < 4; qp++)
#pragma unroll
        for (int m = 0; m < 2; m++) {
            const long long node = base + (qp & 1) * sy + (qp >> 1) * sz + m;
            const float4 r0 = __ldg(g + 3 * node), r1 = __ldg(g + 3 * node + 1), r2 = __ldg(g + 3 * node + 2);
            const float w = (m ? wx : ux) * wyz[qp];
            const float v[9] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x};
#pragma unroll
            for (int c = 0; c < 9; c++) acc[c] += w * v[c];
        }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) G[a][b] = acc[a * 3 + b];
}

__device__ __forceinline__ void gather_grad(const FieldView &f, float x, float y, float z, float G[3][3])
{
    const float cx = fminf(fmaxf(floorf(x), 0.f), f.cmax[0]);
    const float cy = fminf(fmaxf(floorf(y), 0.f), f.cmax[1]);
    const float cz = fminf(fmaxf(floorf(z), 0.f), f.cmax[2]);
    const float wx = x - cx, wy = y - cy, wz = z - cz;
    const long long base = ((long long)small_int(cz) * f.ny + small_int(cy)) * f.nx + small_int(cx);
    gather_grad_cell(f, base, wx, wy, wz, 1.f - wx, 1.f - wy, 1.f - wz, G);
}

// FP32 on a stretched grid: the cell search and Eq. w0 weights of gather_rect
__device__ __forceinline__ void gather_grad_rect(const FieldView &f, float x, float y, float z, float G[3][3])
{
    RectCells<float> rc;
    rect_cells(f, x, y, z, rc);
    const float ux = (rc.r[0].y - x) * rc.r[0].z, uy = (rc.r[1].y - y) * rc.r[1].z, uz = (rc.r[2].y - z) * rc.r[2].z;
    const long long base = ((long long)rc.c[2] * f.ny + rc.c[1]) * f.nx + rc.c[0];
    gather_grad_cell(f, base, 1.f - ux, 1.f - uy, 1.f - uz, ux, uy, uz, G);
}

// FP64: Eq. interp term by term on the 9 gradient components, given the cell
// and the per-axis weights
__device__ __forceinline__ void gather_grad_cell(const FieldView &f, const long long c[3], const double w[3][2],
                                                 double G[3][3])
{
    const long long sy = f.nx, sz = (long long)f.nx * f.ny;
    const long long base = (long long)c[2] * sz + (long long)c[1] * sy + (long long)c[0];
    const double2 *g = (const double2 *)f.grad;
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; k++) acc[k] = 0.0;
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const double wt = w[0][m] * w[1][q] * w[2][p];
                const long long node = base + p * sz + q * sy + m;
                const double2 r0 = __ldg(g + 5 * node), r1 = __ldg(g + 5 * node + 1), r2 = __ldg(g + 5 * node + 2),
                              r3 = __ldg(g + 5 * node + 3), r4 = __ldg(g + 5 * node + 4);
                const double v[9] = {r0.x, r0.y, r1.x, r1.y, r2.x, r2.y, r3.x, r3.y, r4.x};
#pragma unroll
                for (int k = 0; k < 9; k++) acc[k] += wt * v[k];
            }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) G[a][b] = acc[a * 3 + b];
}

__device__ __forceinline__ void gather_grad(const FieldView &f, double x, double y, double z, double G[3][3])
{
    const int cf[3] = {cell_floor64(x, f.nx), cell_floor64(y, f.ny), cell_floor64(z, f.nz)};
    const double xi[3] = {x, y, z};
    long long c[3];
    double w[3][2];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        c[a] = cf[a];
        w[a][0] = int_f64(cf[a] + 1) - xi[a];
        w[a][1] = 1.0 - w[a][0];
    }
    gather_grad_cell(f, c, w, G);
}

// FP64 on a stretched grid: the weights of gather_rect_at
__device__ __forceinline__ void gather_grad_rect(const FieldView &f, double x, double y, double z, double G[3][3])
{
    RectCells<double> rc;
    rect_cells(f, x, y, z, rc);
    const double xi[3] = {x, y, z};
    long long c[3];
    double w[3][2];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double2 cr = rc.r[a];
        c[a] = rc.c[a];
        w[a][0] = (cr.y - xi[a]) / (cr.y - cr.x);
        w[a][1] = 1.0 - w[a][0];
    }
    gather_grad_cell(f, c, w, G);
}

template <typename T, bool RECT = false>
__device__ __forceinline__ bool unit_b(const FieldView &f, T x, T y, T z, T bh[3])
{
    T B[3], J[3];
    gatherg<RECT>(f, x, y, z, B, J, false);
    const T m = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    if (!(m > (T)0) || !(m < (T)INFINITY)) return false;
    bh[0] = B[0] / m;
    bh[1] = B[1] / m;
    bh[2] = B[2] / m;
    return true;
}

// dd: the trial's per-axis scale (step_dd): on a stretched grid way 2 offsets
// +-eps cells of the start cell, eps D_a (FP64 dd = D, FP32 dd = 1/D).
template <typename T, int WAY, bool RECT = false>
__device__ __forceinline__ bool grad_bhat(const FieldView &f, T eps, T x, T y, T z, const T dd[3], T G[3][3])
{
    if constexpr (WAY == 1) {
        if constexpr (RECT) gather_grad_rect(f, x, y, z, G);
        else gather_grad(f, x, y, z, G);
        return true;
    } else {
        const T p[3] = {x, y, z};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            T xp[3] = {p[0], p[1], p[2]}, xm[3] = {p[0], p[1], p[2]};
            T off = eps, span;
            if constexpr (RECT) {
                const T D = sizeof(T) == 8 ? dd[a] : (T)1 / dd[a];
                off = eps * D;
                span = (T)2 * eps * D;
            } else {
                span = (T)2 * eps * (T)f.d[a];
            }
            xp[a] += off;
            xm[a] -= off;
            if constexpr (sizeof(T) == 4) {
                // FP32: divide by the offset the rounded positions realise (their
                // difference is exact); at x ~ 255 cells a float moves in steps
                // of 1.5e-5 cells, 1.5 % of a 0.001-cell offset
                const T h = xp[a] - xm[a];
                span = RECT ? h : h * (T)f.d[a];
            }
            T bp[3], bm[3];
            ok &= unit_b<T, RECT>(f, xp[0], xp[1], xp[2], bp);
            ok &= unit_b<T, RECT>(f, xm[0], xm[1], xm[2], bm);
#pragma unroll
            for (int b = 0; b < 3; b++) G[a][b] = (bp[b] - bm[b]) / span;
        }
        return ok;
    }
}

// fourth root through the correctly rounded square root
__device__ __forceinline__ float root4(float v) { return sqrtf(sqrtf(v)); }
__device__ __forceinline__ double root4(double v) { return sqrt(sqrt(v)); }

// the tolerance (RKF45) or step (fixed-step scheme) of a line in the
// perpendicular case: rotated seeds, their extra lines, Method II, seed lists
__device__ __forceinline__ double ctl_perp(const DevParams &p) { return p.scheme == 1 ? p.step : p.tol; }

// x^e for the obliquity factor of Eq. tol (x sqrt(x) for the usual e = 1.5)
__device__ __forceinline__ double obliq_pow(double x, double e) { return e == 1.5 ? x * sqrt(x) : pow(x, e); }

// physical coordinate of an index coordinate, without contraction so that the
// value matches a plain multiply-then-add
__device__ __forceinline__ double to_phys(double o, double d, double xi) { return __dadd_rn(o, __dmul_rn(d, xi)); }

// physical coordinate of a state coordinate (the FP64 state on a stretched
// grid is physical already)
template <typename T, bool RECT>
__device__ __forceinline__ double phys_of(const FieldView &f, double x, int a)
{
    if constexpr (RECT && sizeof(T) == 8) return x;
    else return to_phys(f.o[a], f.d[a], x);
}

// the box bounds in double state coordinates (for seeds; the FP32 tracer's
// float bounds are these rounded, so a seed inside stays inside)
template <typename T, bool RECT>
__device__ __forceinline__ double dlo(const FieldView &f, int a)
{
    return (RECT && sizeof(T) == 8) ? f.lo64[a] : 0.0;
}

template <typename T, bool RECT>
__device__ __forceinline__ double dhi(const FieldView &f, int a)
{
    if constexpr (RECT) return sizeof(T) == 8 ? f.hi64[a] : f.hi64[a] - f.lo64[a];
    else return (double)(axis_n(f, a) - 1);
}

// a state position (double) inside the closed box
template <typename T, bool RECT>
__device__ __forceinline__ bool in_box(const FieldView &f, const double xi[3])
{
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; a++) in = in && xi[a] >= dlo<T, RECT>(f, a) && xi[a] <= dhi<T, RECT>(f, a);
    return in;
}

template <typename T>
__device__ __forceinline__ T sel3(int a, T v0, T v1, T v2)
{
    return a == 0 ? v0 : (a == 1 ? v1 : v2);
}

// Seed position of lattice index (i, j, k) in physical coordinates, evaluated
// as o + t1 + t2 + t3 left to right without contraction.
__device__ __forceinline__ void lattice_seed(const Lattice &L, long long i, long long j, long long k, double r[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double v = __dadd_rn(L.o[a], __dmul_rn((double)i + 0.5, L.a1[a]));
        v = __dadd_rn(v, __dmul_rn((double)j + 0.5, L.a2[a]));
        v = __dadd_rn(v, __dmul_rn((double)k + 0.5, L.a3[a]));
        r[a] = v;
    }
}

// Orthonormal u, v perpendicular to bhat: u = unit(bhat x e_m) with m the axis
// of smallest |bhat_m| (lowest index on ties), v = bhat x u.
__device__ __forceinline__ void perp_frame(const double bh[3], double u[3], double v[3])
{
    int m = 0;
    if (fabs(bh[1]) < fabs(bh[m])) m = 1;
    if (fabs(bh[2]) < fabs(bh[m])) m = 2;
    const double e[3] = {m == 0 ? 1.0 : 0.0, m == 1 ? 1.0 : 0.0, m == 2 ? 1.0 : 0.0};
    const double t[3] = {bh[1] * e[2] - bh[2] * e[1], bh[2] * e[0] - bh[0] * e[2], bh[0] * e[1] - bh[1] * e[0]};
    const double nt = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    u[0] = t[0] / nt;
    u[1] = t[1] / nt;
    u[2] = t[2] / nt;
    v[0] = bh[1] * u[2] - bh[2] * u[1];
    v[1] = bh[2] * u[0] - bh[0] * u[2];
    v[2] = bh[0] * u[1] - bh[1] * u[0];
}

// B at a state position in double (for seeds, frames and end normals)
template <typename T, bool RECT = false>
__device__ __forceinline__ void b_at(const FieldView &f, double x, double y, double z, double B[3])
{
    T Bt[3], Jt[3];
    gatherg<RECT>(f, (T)x, (T)y, (T)z, Bt, Jt, false);
    B[0] = (double)Bt[0];
    B[1] = (double)Bt[1];
    B[2] = (double)Bt[2];
}

// ---------------------------------------------------------------------------
// lane state
// ---------------------------------------------------------------------------
template <typename T>
struct Lane {
    long long line;   // record index
    T x, y, z;        // current position (cells)
    T sx, sy, sz;     // seed position
    T h;              // current step
    T s0;             // end 1 is traced along -s0 B
    T ox, oy, oz;     // end of the exiting step (chord fallback)
    T t0;             // chord parameter of the first crossed face
    double tol;          // FP64: the line's tolerance; FP32: its square
    float tolf2;         // FP32: tol^2 for the step factor
    double lacc, twacc;  // length / Tw of the current direction (FP64 sums)
    float ls, lc, ts, tc;  // the same as compensated FP32 sums and their carries
    double l1, tw1;      // totals of end 1
    double ol, otw;      // exiting step: FP64 sums at its end / FP32 its increments
    int steps, st, end, mode, hface, tries, fc0;
    int tcur, tn;        // step tape: current chunk (-1 none yet, -2 pool exhausted), steps in it
    // Method II: deviation vectors (current, at the seed, at the end of the exiting step)
    T u[3], v[3], u0[3], v0[3], ou[3], ov[3];
};

// Length and Tw of the current direction: FP64 sums (ACC, and the FP64
// tracer) or compensated FP32 sums (Kahan 1965) whose total is formed in FP64
// once per direction.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <typename T, bool ACC>
__device__ __forceinline__ void acc_reset(Lane<T> &L)
{
    if (ACC) {
        L.lacc = 0.0;
        L.twacc = 0.0;
    } else {
        L.ls = L.lc = L.ts = L.tc = 0.f;
    }
}

template <typename T, bool ACC>
__device__ __forceinline__ void acc_add(Lane<T> &L, T dl, T dtw)
{
    if (ACC) {
        L.lacc = L.lacc + (double)dl;
        L.twacc = L.twacc + (double)dtw;
    } else {
        kahan_add(L.ls, L.lc, (float)dl);
        kahan_add(L.ts, L.tc, (float)dtw);
    }
}

template <typename T, bool ACC>
__device__ __forceinline__ double acc_len(const Lane<T> &L)
{
    return ACC ? L.lacc : (double)L.ls - (double)L.lc;
}

template <typename T, bool ACC>
__device__ __forceinline__ double acc_tw(const Lane<T> &L)
{
    return ACC ? L.twacc : (double)L.ts - (double)L.tc;
}

// FP64 end record: physical footpoint, face and Bn.
template <typename T>
__device__ __forceinline__ void write_end(const TraceArgs &A, const LineRecs &R, const Lane<T> &L, int e,
                                          double px, double py, double pz, int face, double bn)
{
    double *r = (e == 0 ? R.r1 : R.r2) + 3 * L.line;
    r[0] = px;
    r[1] = py;
    r[2] = pz;
    (e == 0 ? R.f1 : R.f2)[L.line] = (int8_t)face;
    double *bnp = (e == 0 ? R.bn1 : R.bn2);
    if (bnp) bnp[L.line] = bn;
}

// FP32 end record: index-space footpoint and face (the assembly forms the
// physical footpoint and Bn).
__device__ __forceinline__ void write_end32(const LineRecs &R, long long line, int e, float x, float y, float z,
                                            int face)
{
    float *r = (e == 0 ? R.xi1 : R.xi2) + 3 * line;
    r[0] = x;
    r[1] = y;
    r[2] = z;
    (e == 0 ? R.f1 : R.f2)[line] = (int8_t)face;
}

// ---------------------------------------------------------------------------
// step tape (adjoint forward pass; see Tape)
// ---------------------------------------------------------------------------
// 16-byte vector stores of the kept states and stage derivatives (addresses
// 16-byte aligned: the arrays are, and their strides are multiples of 16 B).
__device__ __forceinline__ void store_state(float *p, float x, float y, float z)
{
    *(float4 *)p = make_float4(x, y, z, 0.f);
}
__device__ __forceinline__ void store_state(double *p, double x, double y, double z)
{
    ((double2 *)p)[0] = make_double2(x, y);
    ((double2 *)p)[1] = make_double2(z, 0.0);
}
// the first N (a multiple of 4) values of v
template <typename T, int N>
__device__ __forceinline__ void store_vec(T *p, const T v[])
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < N; q += 4) *(float4 *)(p + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < N; q += 2) *(double2 *)(p + q) = make_double2(v[q], v[q + 1]);
    }
}

// Open a new chunk whose checkpoint is the current state. Returns false when
// the pool is exhausted (the half-line is then no longer taped).
template <typename T>
__device__ __forceinline__ bool tape_chunk(const Tape &tp, Lane<T> &L)
{
    const unsigned long long c = atomicAdd(tp.next, 1ull);
    if (c >= (unsigned long long)tp.cap) {
        L.tcur = -2;
        return false;
    }
    tp.prev[c] = L.tcur;
    tp.owner[c] = (int32_t)(tp.hl_base + 2 * L.line + L.end);
    T *x = (T *)tp.xi + 4 * c;
    x[0] = L.x;
    x[1] = L.y;
    x[2] = L.z;
    x[3] = (T)0;
    if (tp.wx && (long long)c < tp.wcap) store_state((T *)tp.wx + c * (long long)(tp.k + 1) * kStateStride, L.x, L.y, L.z);
    L.tcur = (int)c;
    L.tn = 0;
    return true;
}

// An accepted step of size h from the current state; ns stages' position
// derivatives k0, k1, k2 and the end state (x1, y1, z1) are kept too when the
// tape holds them (Tape::wx, wk).
template <typename T, int NS>
__device__ __forceinline__ void tape_step(const Tape &tp, Lane<T> &L, T h, const T k0[], const T k1[], const T k2[],
                                          T x1, T y1, T z1)
{
    if (L.tcur == -2) return;
    if ((L.tcur < 0 || L.tn == tp.k) && !tape_chunk(tp, L)) return;
    const long long j = (long long)L.tcur * tp.k + L.tn;
    ((T *)tp.h)[j] = h;
    if (tp.wx && L.tcur < tp.wcap) {
        T v[kStageStride];
#pragma unroll
        for (int s = 0; s < NS; s++) {
            v[3 * s + 0] = k0[s];
            v[3 * s + 1] = k1[s];
            v[3 * s + 2] = k2[s];
        }
#pragma unroll
        for (int q = 3 * NS; q < kStageStride; q++) v[q] = (T)0;
        store_vec<T, (3 * NS + 3) / 4 * 4>((T *)tp.wk + j * kStageStride, v);
        store_state((T *)tp.wx + ((long long)L.tcur * (tp.k + 1) + L.tn + 1) * kStateStride, x1, y1, z1);
    }
    L.tn++;
}

// The current direction ends at (x, y, z) by end code `code` (hx: the
// exiting step of a chord end).
template <typename T>
__device__ __forceinline__ void tape_end(const Tape &tp, Lane<T> &L, int code, T x, T y, T z, T hx)
{
    if (L.tcur == -1) tape_chunk(tp, L);  // no accepted step: the checkpoint is the seed
    const long long hl = tp.hl_base + 2 * L.line + L.end;
    const int sg = (L.end == 0) == (L.s0 > (T)0) ? -1 : 1;
    tp.head[hl] = make_int4(L.tcur, L.tn, L.tcur >= 0 ? code : -2, sg);
    T *e = (T *)tp.xe + 4 * hl;
    e[0] = x;
    e[1] = y;
    e[2] = z;
    e[3] = hx;
}

// Split directions (the taped tracer): each direction of a line is its own
// work item, so the line's status bits, trial count and (FP64) length/Tw sums
// are combined with atomics on records cleared before the launch. Each
// direction finishes with its share; the one that completes the trial count
// marks the line MAXSTEPS if both together used more than max_steps. (A sum of
// two values onto zero does not depend on their order.)
__device__ __forceinline__ void or_status(uint8_t *st, long long line, unsigned bits)
{
    unsigned *w = (unsigned *)(st + (line & ~3LL));
    atomicOr(w, bits << (8 * (unsigned)(line & 3)));
}

template <typename T>
__device__ __forceinline__ void split_finish(const TraceArgs &A, const LineRecs &R, Lane<T> &L, bool bad)
{
    const int before = atomicAdd(R.steps + L.line, L.steps);
    unsigned st = (unsigned)L.st;
    if ((long long)before + L.steps > A.p.max_steps) {
        st |= FQSL_LINE_MAXSTEPS;
        bad = true;
    }
    or_status(R.st, L.line, st);
    if constexpr (sizeof(T) == 8) {
        if (bad) {
            if (R.tw) R.tw[L.line] = NAN;
            if (R.len) R.len[L.line] = NAN;
        }
    }
}

// Finish the line with a bad status (MAXSTEPS or NULL_B): the unfinished end
// is the current position, an untraced end the seed, their faces -1.
template <typename T, bool SPLIT = false, bool RECT = false>
__device__ __forceinline__ void finish_bad(const TraceArgs &A, const LineRecs &R, Lane<T> &L, unsigned bit)
{
    const FieldView &f = A.f;
    L.st |= bit;
    if constexpr (sizeof(T) == 8) {
        write_end(A, R, L, L.end, phys_of<T, RECT>(f, (double)L.x, 0), phys_of<T, RECT>(f, (double)L.y, 1),
                  phys_of<T, RECT>(f, (double)L.z, 2), -1, 0.0);
        if (L.end == 0 && !SPLIT)
            write_end(A, R, L, 1, phys_of<T, RECT>(f, (double)L.sx, 0), phys_of<T, RECT>(f, (double)L.sy, 1),
                      phys_of<T, RECT>(f, (double)L.sz, 2), -1, 0.0);
        if (R.tw) R.tw[L.line] = NAN;
        if (R.len) R.len[L.line] = NAN;
    } else {
        write_end32(R, L.line, L.end, (float)L.x, (float)L.y, (float)L.z, -1);
        if (L.end == 0 && !SPLIT) write_end32(R, L.line, 1, (float)L.sx, (float)L.sy, (float)L.sz, -1);
    }
    if constexpr (SPLIT) {
        split_finish(A, R, L, true);
    } else {
        R.st[L.line] = (uint8_t)L.st;
        R.steps[L.line] = L.steps;
    }
}

// A direction reached a face at index position (x, y, z) with deviation
// vectors (du, dv) (Method II only).
template <typename T, bool ACC, int DEV = 0, bool SPLIT = false, bool RECT = false>
__device__ __forceinline__ bool finish_dir(const TraceArgs &A, const LineRecs &R, Lane<T> &L, T x, T y, T z,
                                           int face, const T *du = nullptr, const T *dv = nullptr)
{
    const FieldView &f = A.f;
    if constexpr (DEV != 0) {
        if constexpr (sizeof(T) == 8) {
            double *d = R.dev64 + 12 * L.line + 6 * L.end;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                d[c] = du[c];
                d[3 + c] = dv[c];
            }
        } else {
            float *d = R.dev32 + 12 * L.line + 6 * L.end;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                d[c] = du[c];
                d[3 + c] = dv[c];
            }
        }
    }
    if constexpr (sizeof(T) == 8) {
        double B[3];
        b_at<T, RECT>(f, (double)x, (double)y, (double)z, B);
        const int ax = face >> 1;
        write_end(A, R, L, L.end, phys_of<T, RECT>(f, (double)x, 0), phys_of<T, RECT>(f, (double)y, 1),
                  phys_of<T, RECT>(f, (double)z, 2), face, sel3<double>(ax, B[0], B[1], B[2]));
        if (R.be64) {
            double *be = R.be64 + 6 * L.line + 3 * L.end;
            be[0] = B[0];
            be[1] = B[1];
            be[2] = B[2];
        }
    } else {
        write_end32(R, L.line, L.end, (float)x, (float)y, (float)z, face);
        if (R.kacc) {
            float4 k;
            if (ACC) {
                // FP64 sums: carry the value and its float residue
                const float lh = (float)L.lacc, th = (float)L.twacc;
                k = make_float4(lh, -(float)(L.lacc - (double)lh), th, -(float)(L.twacc - (double)th));
            } else {
                k = make_float4(L.ls, L.lc, L.ts, L.tc);
            }
            R.kacc[2 * L.line + L.end] = k;
        }
    }
    if constexpr (SPLIT) {
        if constexpr (sizeof(T) == 8) {
            if (R.tw) atomicAdd(R.tw + L.line, acc_tw<T, ACC>(L));
            if (R.len) atomicAdd(R.len + L.line, acc_len<T, ACC>(L));
        }
        split_finish(A, R, L, false);
        return false;
    }
    if (L.end == 0) {
        if constexpr (sizeof(T) == 8) {
            L.l1 = acc_len<T, ACC>(L);
            L.tw1 = acc_tw<T, ACC>(L);
        }
        L.end = 1;
        L.x = L.sx;
        L.y = L.sy;
        L.z = L.sz;
        if constexpr (DEV != 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                L.u[c] = L.u0[c];
                L.v[c] = L.v0[c];
            }
        }
        L.h = A.p.scheme == 1 ? (T)L.tol : (T)A.p.h0;  // fixed step: the line's step (in tol)
        L.mode = 0;
        L.tcur = -1;
        L.tn = 0;
        acc_reset<T, ACC>(L);
        return true;
    }
    R.st[L.line] = (uint8_t)L.st;
    R.steps[L.line] = L.steps;
    if constexpr (sizeof(T) == 8) {
        if (R.tw) R.tw[L.line] = L.tw1 + acc_tw<T, ACC>(L);
        if (R.len) R.len[L.line] = L.l1 + acc_len<T, ACC>(L);
    }
    return false;
}

template <typename T, bool RECT = false>
__device__ __forceinline__ bool inside(const FieldView &f, T x, T y, T z)
{
    if constexpr (RECT)
        return x >= lo_of<T, RECT>(f, 0) && x <= hi_of<T, RECT>(f, 0) && y >= lo_of<T, RECT>(f, 1) &&
               y <= hi_of<T, RECT>(f, 1) && z >= lo_of<T, RECT>(f, 2) && z <= hi_of<T, RECT>(f, 2);
    else
        return x >= (T)0 && x <= (T)(f.nx - 1) && y >= (T)0 && y <= (T)(f.ny - 1) && z >= (T)0 &&
               z <= (T)(f.nz - 1);
}

// Start a line at index position xi (FP64: (r0 - o)/d as written) with
// orientation vector n (NULL: end 1 is the backward end) and tolerance tol
// (with the fixed-step scheme: its step). Returns false if the line ends at
// once (outside / null).
template <typename T, bool ACC, bool RECT = false>
__device__ __forceinline__ bool start_line(const TraceArgs &A, const LineRecs &R, Lane<T> &L, const double xi[3],
                                           const double *n, double tol, int st0)
{
    const FieldView &f = A.f;
    constexpr bool kF64 = sizeof(T) == 8;
    L.sx = (T)xi[0];
    L.sy = (T)xi[1];
    L.sz = (T)xi[2];
    L.x = L.sx;
    L.y = L.sy;
    L.z = L.sz;
    L.st = st0;
    L.steps = 0;
    L.end = 0;
    L.mode = 0;
    L.tcur = -1;
    L.tn = 0;
    acc_reset<T, ACC>(L);
    L.h = (T)A.p.h0;
    if (A.p.scheme == 1) {
        // fixed-step scheme: tol carries the line's step
        L.tol = tol;
        L.h = (T)tol;
    } else if (kF64) {
        L.tol = tol;
    } else {
        L.tol = tol * tol;
        L.tolf2 = (float)L.tol;
    }
    const bool in = in_box<T, RECT>(f, xi);
    unsigned bad = 0;
    T B0[3] = {0, 0, 0};
    if (!in) {
        bad = FQSL_LINE_OUTSIDE;
    } else {
        T J0[3], dd[3];
        gatherg<RECT>(f, L.sx, L.sy, L.sz, B0, J0, false);
        step_dd<T, RECT>(f, L.sx, L.sy, L.sz, dd);
        T bb;
        if (kF64) {
            const T b0 = B0[0] / dd[0], b1 = B0[1] / dd[1], b2 = B0[2] / dd[2];
            bb = b0 * b0 + b1 * b1 + b2 * b2;
        } else {
            const T b0 = B0[0] * dd[0], b1 = B0[1] * dd[1], b2 = B0[2] * dd[2];
            bb = b0 * b0 + b1 * b1 + b2 * b2;
        }
        if (!(bb > (T)0) || !(bb < (T)INFINITY)) bad = FQSL_LINE_NULL_B;
    }
    if (bad) {
        L.st |= bad;
        // footpoints of a line that never started: its seed
        if constexpr (sizeof(T) == 8) {
            const double qx = phys_of<T, RECT>(f, xi[0], 0), qy = phys_of<T, RECT>(f, xi[1], 1),
                         qz = phys_of<T, RECT>(f, xi[2], 2);
            write_end(A, R, L, 0, qx, qy, qz, -1, 0.0);
            write_end(A, R, L, 1, qx, qy, qz, -1, 0.0);
            if (R.tw) R.tw[L.line] = NAN;
            if (R.len) R.len[L.line] = NAN;
        } else {
            write_end32(R, L.line, 0, (float)xi[0], (float)xi[1], (float)xi[2], -1);
            write_end32(R, L.line, 1, (float)xi[0], (float)xi[1], (float)xi[2], -1);
        }
        R.st[L.line] = (uint8_t)L.st;
        R.steps[L.line] = 0;
        return false;
    }
    L.s0 = (T)1;
    if (n && (B0[0] * (T)n[0] + B0[1] * (T)n[1] + B0[2] * (T)n[2] < (T)0)) L.s0 = (T)-1;
    return true;
}

// Lattice seed: frame, tolerance and rotation decision (Sec. 4). reg_rot:
// queue a rotated seed for its extra lines (once per seed).
template <typename T, bool ACC, int DEV = 0, bool RECT = false>
__device__ __forceinline__ bool init_lattice(const TraceArgs &A, Lane<T> &L, long long item, bool reg_rot = true)
{
    constexpr bool kF64 = sizeof(T) == 8;
    const Lattice &G = A.lat;
    const long long per_tile = kTileU * kTileV;
    const long long w = item % per_tile;
    long long t = item / per_tile;
    const long long tu = t % G.tiles_u;
    t /= G.tiles_u;
    const long long tv = t % G.tiles_v;
    const long long k = t / G.tiles_v;
    const long long i = tu * kTileU + (w % kTileU);
    const long long j = tv * kTileV + (w / kTileU);
    if (i >= G.n1 || j >= G.n2 || k >= G.n3) return false;
    const long long idx = i + G.n1 * (j + G.n2 * k);
    L.line = idx;
    const FieldView &f = A.f;
    const LineRecs &R = A.rec;
    if constexpr (!kF64) {
        // FP32: the seed pre-pass did the set-up (and wrote final records of
        // seeds outside the box or on a null)
        const uint8_t fl = A.prep.flags[idx];
        if (fl & kSeedDone) return false;
        const float4 sd = A.prep.seed[idx];
        L.sx = L.x = sd.x;
        L.sy = L.y = sd.y;
        L.sz = L.z = sd.z;
        L.tolf2 = sd.w;
        L.tol = (double)sd.w;
        L.s0 = (fl & kSeedNegS0) ? (T)-1 : (T)1;
        L.st = (fl & kSeedRotated) ? FQSL_LINE_ROTATED : 0;
        L.steps = 0;
        L.end = 0;
        L.mode = 0;
        L.tcur = -1;
        L.tn = 0;
        acc_reset<T, ACC>(L);
        L.h = A.p.scheme == 1 ? (T)sd.w : (T)A.p.h0;  // fixed step: the pre-pass's step
        if constexpr (DEV != 0) {
            const float4 fu = A.prep.fu[idx], fv = A.prep.fv[idx];
            L.u[0] = L.u0[0] = fu.x;
            L.u[1] = L.u0[1] = fu.y;
            L.u[2] = L.u0[2] = fu.z;
            L.v[0] = L.v0[0] = fv.x;
            L.v[1] = L.v0[1] = fv.y;
            L.v[2] = L.v0[2] = fv.z;
        }
        return true;
    }
    double xi[3];
    if (kF64) {
        // physical seed, then (r0 - o)/d, as written (the physical seed itself
        // on a stretched grid)
        double r0[3];
        lattice_seed(G, i, j, k, r0);
#pragma unroll
        for (int a = 0; a < 3; a++) xi[a] = state_of<T, RECT>(f, r0[a], a);
    } else {
        const double fi = (double)i + 0.5, fj = (double)j + 0.5, fk = (double)k + 0.5;
#pragma unroll
        for (int a = 0; a < 3; a++) xi[a] = fma(fk, G.xa3[a], fma(fj, G.xa2[a], fma(fi, G.xa1[a], G.xo[a])));
    }
    // B at the seed, S0 obliquity and tolerance (fixed-step scheme: step)
    double tol = ctl_perp(A.p);
    int st0 = 0;
    double bn0 = 0.0;
    const bool in = in_box<T, RECT>(f, xi);
    if (in) {
        T B0[3], J0[3];
        gatherg<RECT>(f, (T)xi[0], (T)xi[1], (T)xi[2], B0, J0, false);
        const T nB = sqrt(B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2]);
        if (nB > (T)0 && nB < (T)INFINITY) {
            const T bn = B0[0] * (T)G.n0[0] + B0[1] * (T)G.n0[1] + B0[2] * (T)G.n0[2];
            if (A.p.method == 2) {
                bn0 = (double)nB;
            } else {
                const T ratio = fabs(bn) / nB;
                bool on_face = false;
                if (G.normal_axis >= 0) {
                    const double xa = xi[G.normal_axis];
                    on_face = (xa == dlo<T, RECT>(f, G.normal_axis)) || (xa == dhi<T, RECT>(f, G.normal_axis));
                }
                if (G.allow_rot && ratio < (T)A.p.rot && !on_face) {
                    st0 = FQSL_LINE_ROTATED;
                    bn0 = (double)nB;
                    if (reg_rot) {
                        const unsigned slot = atomicAdd(A.q.rot_count, 1u);
                        A.q.rot_seed[slot] = (int32_t)idx;
                        A.q.rot_slot[idx] = (int32_t)slot + 1;
                    }
                } else {
                    bn0 = (double)bn;
                    if (A.p.scheme == 1) {
                        tol = fmax(A.p.step * (double)ratio, A.p.step_min);  // Eq. step
                    } else if (kF64) {
                        tol = A.p.tol * obliq_pow(fmax((double)ratio, A.p.rot), A.p.texp);
                    } else {
                        const float x = fmaxf((float)ratio, (float)A.p.rot);
                        const float g = A.p.texp == 1.5 ? x * sqrtf(x) : __powf(x, (float)A.p.texp);
                        tol = A.p.tol * (double)g;
                    }
                }
            }
        }
    }
    R.bn0[idx] = bn0;
    const bool started = start_line<T, ACC, RECT>(A, R, L, xi, G.n0, tol, st0);
    if constexpr (DEV != 0) {
        if (started) {
            // S0 perpendicular to B: U0, V0 = the frame of B/|B| at the seed (Sec. 4)
            double B0[3], u[3], v[3];
            b_at<T, RECT>(f, xi[0], xi[1], xi[2], B0);
            const double nB = sqrt(B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2]);
            const double bh[3] = {B0[0] / nB, B0[1] / nB, B0[2] / nB};
            perp_frame(bh, u, v);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                L.u[c] = L.u0[c] = (T)u[c];
                L.v[c] = L.v0[c] = (T)v[c];
            }
        }
    }
    return started;
}

// Rotated extra line q (0: +u, 1: -u, 2: +v, 3: -v) of rotated slot s (Sec. 4).
template <typename T, bool ACC, bool RECT = false>
__device__ __forceinline__ bool init_extra(const TraceArgs &A, Lane<T> &L, long long item)
{
    const Lattice &G = A.lat;
    const long long s = item >> 2;
    const int q = (int)(item & 3);
    const long long idx = A.q.rot_seed[s];
    const long long i = idx % G.n1, j = (idx / G.n1) % G.n2, k = idx / (G.n1 * G.n2);
    double r0[3];
    lattice_seed(G, i, j, k, r0);
    const FieldView &f = A.f;
    double xi[3], B0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) xi[a] = state_of<T, RECT>(f, r0[a], a);
    b_at<T, RECT>(f, xi[0], xi[1], xi[2], B0);
    const double nB = sqrt(B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2]);
    double bh[3] = {B0[0] / nB, B0[1] / nB, B0[2] / nB}, u[3], v[3];
    perp_frame(bh, u, v);
    const double sc = (B0[0] * G.n0[0] + B0[1] * G.n0[1] + B0[2] * G.n0[2] < 0.0) ? -1.0 : 1.0;
    const double nrot[3] = {sc * bh[0], sc * bh[1], sc * bh[2]};
    const double *dir = (q < 2) ? u : v;
    const double sg = (q & 1) ? -1.0 : 1.0;
    double rr[3];
#pragma unroll
    for (int a = 0; a < 3; a++) rr[a] = r0[a] + sg * G.drot * dir[a];
    double xr[3];
#pragma unroll
    for (int a = 0; a < 3; a++) xr[a] = state_of<T, RECT>(f, rr[a], a);
    L.line = item;
    return start_line<T, ACC, RECT>(A, A.ext, L, xr, nrot, ctl_perp(A.p), 0);
}

template <typename T, bool ACC, bool RECT = false>
__device__ __forceinline__ bool init_list(const TraceArgs &A, Lane<T> &L, long long item)
{
    L.line = item;
    const FieldView &f = A.f;
    double xi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) xi[a] = state_of<T, RECT>(f, A.seeds[3 * item + a], a);
    return start_line<T, ACC, RECT>(A, A.rec, L, xi, nullptr, ctl_perp(A.p), 0);
}

// ---------------------------------------------------------------------------
// the persistent kernel body
// ---------------------------------------------------------------------------
// ACC: FP64 sums for the error norm and for length/Tw (always true for the
// FP64 tracer); false: FP32 error norm and compensated FP32 sums.
// DEV: 0 = positions only (Method I, twist); 1, 2 = Method II deviation
// vectors with grad(B/|B|) by way 1 or way 2 (lattice source only).
// BATCH: the launch traces the entries of a batch (BatchArgs); each lane keeps
// the entry of its line. A0 holds the launch-wide parameters and counter.
// TAPE: also write the step tape A0.tape (Method I). Lattice lines are then
// traced with their two directions as separate work items (twice the
// lattice's items; see split_finish) so that a long line's halves run side by
// side; the extra lines of rotated seeds keep one item per line.
// RECT: the field is on a stretched grid (FieldView::rect; Method I and
// twist lists): positions are physical (FP32: relative to the first node),
// cells are searched, and each trial scales its step and error by the widths
// of the cell it starts in (Sec. 2.3).
// SCH: 0 = RKF45, 1 = the fixed-step 3/8 rule (every trial accepted; the
// line's step is held in L.h, halved only by a grazing exit).
template <typename T, int SRC, bool ACC, int DEV = 0, bool BATCH = false, bool TAPE = false, bool RECT = false,
          int SCH = 0>
__device__ __forceinline__ void trace_body(const TraceArgs &A0, const BatchArgs &BA)
{
    constexpr bool SPLIT = TAPE && SRC == kSrcLattice;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    constexpr bool kF64 = sizeof(T) == 8;
    const T hmin = (T)A0.p.hmin, hmax = (T)A0.p.hmax;
    const T graze = (T)A0.p.graze;
    const int max_steps = (int)A0.p.max_steps;

    long long nitems = A0.nitems;
    if (BATCH) nitems = BA.ibase[BA.nent];
    else if (SRC == kSrcExtra) nitems = 4LL * (long long)(*(volatile unsigned *)A0.q.rot_count);

    long long ck_cur = 0, ck_end = 0, ck_base = 0;
    int ck_ent = 0;
    bool exhausted = false;
    bool active = false;
    bool waiting = false;  // sync_dirs: first direction done, second not started
    int eb = 0;            // BATCH: entry of this lane's line
    Lane<T> L;
    L.line = 0;
    // the entry of this lane's line (the launch itself when not batched)
    auto ent = [&]() -> const TraceArgs & {
        if constexpr (BATCH) return BA.desc[eb];
        else return A0;
    };

    for (;;) {
        // refill idle lanes from the warp's chunk / the global counter, once
        // at least p.refill lanes are idle (or none is busy)
        unsigned idle = __ballot_sync(FULL, !active);
        const bool refill = __popc(idle) >= A0.p.refill || idle == FULL;
        while (refill && idle != 0u && !exhausted) {
            if (ck_cur >= ck_end) {
                unsigned long long base = 0;
                const long long chunk = BATCH ? (long long)kChunk : (long long)A0.p.chunk;
                if (lane == 0) base = atomicAdd(A0.q.head, (unsigned long long)chunk);
                base = __shfl_sync(FULL, base, 0);
                if ((long long)base >= nitems) {
                    exhausted = true;
                    break;
                }
                ck_cur = (long long)base;
                ck_end = min(ck_cur + chunk, nitems);
                ck_base = 0;
                if constexpr (BATCH) {
                    // entry holding this chunk (chunks never span entries)
                    int lo = 0, hi = BA.nent - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (BA.ibase[mid] <= ck_cur) lo = mid;
                        else hi = mid - 1;
                    }
                    ck_ent = lo;
                    ck_base = BA.ibase[lo];
                }
            }
            const long long avail = ck_end - ck_cur;
            const int rank = __popc(idle & lt_mask);
            if (!active && rank < avail) {
                const long long item = ck_cur + rank - ck_base;
                eb = ck_ent;
                const TraceArgs &E = ent();
                if (SRC == kSrcLattice) {
                    if constexpr (SPLIT) {
                        // items come in 32-lane groups: a tile's direction 0,
                        // then the same tile's direction 1
                        const long long g = item >> 5;
                        active = init_lattice<T, ACC, DEV, RECT>(E, L, ((g >> 1) << 5) | (item & 31), (g & 1) == 0);
                        if (active && (g & 1)) L.end = 1;
                    } else {
                        active = init_lattice<T, ACC, DEV, RECT>(E, L, item);
                    }
                }
                else if (SRC == kSrcExtra)
                    active = item < 4LL * (long long)*E.q.rot_count && init_extra<T, ACC, RECT>(E, L, item);
                else active = init_list<T, ACC, RECT>(E, L, item);
            }
            ck_cur += min((long long)__popc(idle), avail);
            idle = __ballot_sync(FULL, !active);
        }
        if (__ballot_sync(FULL, active) == 0u) break;
        if (A0.p.sync_dirs) {
            // lanes that finished their first direction wait until none is left in it
            if (__ballot_sync(FULL, active && !waiting && L.end == 0) == 0u) waiting = false;
        }
        if (!active || waiting) continue;

        const TraceArgs &A = ent();
        const FieldView &f = A.f;
        const LineRecs &R = (SRC == kSrcExtra) ? A.ext : A.rec;
        // FP32 multiplies by 1/d, FP64 divides by d (see rhs); on a stretched
        // grid d is the width of the start point's cell
        T dd[3];
        RectCells<T> rc0;  // stretched grid: the start point's cells (the first stage is there too)
        if constexpr (RECT) {
            rect_cells(f, L.x, L.y, L.z, rc0);
            dd_of(rc0, dd);
        } else {
            step_dd<T, RECT>(f, L.x, L.y, L.z, dd);
        }

        // ---- one trial: normal RKF45 step or exit (Henon) step ----
        const bool henon = L.mode != 0;
        const int hax = L.hface >> 1;
        const int hmaxside = L.hface & 1;
        const T hsign = hmaxside ? (T)1 : (T)-1;
        const T target = hmaxside ? hi_of<T, RECT>(f, hax) : lo_of<T, RECT>(f, hax);
        const T sgn = (L.end == 0) ? -L.s0 : L.s0;
        T hh;
        if (!henon) {
            if (L.steps >= max_steps) {
                finish_bad<T, SPLIT, RECT>(A, R, L, FQSL_LINE_MAXSTEPS);
                active = false;
                continue;
            }
            hh = L.h;
        } else {
            hh = target - sel3<T>(hax, L.x, L.y, L.z);
        }
        L.steps++;

        constexpr int NS = DEV ? 11 : 5;  // xi (3), length, Tw [, U (3), V (3)]
        T k0[5], k1[5], k2[5];  // position derivatives of stages 1..5
        T kd[DEV ? 5 : 1][6];   // deviation derivatives of stages 1..5 (Method II)
        T a4[3] = {0, 0, 0}, a5[3] = {0, 0, 0};  // FP64: 5th-order sums; FP32: 5th - 4th
        T ad[6] = {0, 0, 0, 0, 0, 0};           // Method II: 4th-order sums of U, V
        T l4 = 0, tw4 = 0;
        int fail = 0;  // first failing stage: 1 null field, 2 grazing exit step
        constexpr int NST = Tab<T, SCH>::N;
#pragma unroll
        for (int s = 0; s < NST; s++) {
            T px = 0, py = 0, pz = 0;
#pragma unroll
            for (int r = 0; r < s; r++) {
                const T c = Tab<T, SCH>::a(s, r);
                px += c * k0[r];
                py += c * k1[r];
                pz += c * k2[r];
            }
            px = L.x + hh * px;
            py = L.y + hh * py;
            pz = L.z + hh * pz;
            T o[NS];
            // FP32: RKF45's stages 1 and 5 have zero 4th-order weight, so their
            // Tw integrand is not formed (nor their curl B loaded)
            const bool wj = kF64 || SCH != 0 || (s != 1 && s != 5);
            bool ok = rhsg<RECT>(f, dd, sgn, px, py, pz, o, (RECT && s == 0) ? &rc0 : nullptr, wj);
            if constexpr (DEV != 0) {
                // stage deviation vectors and Eq. rb2: dU/dtau = sigma (ds/dtau) (U . grad)(B/|B|)
                T us[6];
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    T acc = 0;
#pragma unroll
                    for (int r = 0; r < s; r++) acc += Tab<T, SCH>::a(s, r) * kd[r][c];
                    us[c] = (c < 3 ? L.u[c] : L.v[c - 3]) + hh * acc;
                }
                T G[3][3];
                ok = grad_bhat<T, DEV, RECT>(f, (T)A0.p.eps2, px, py, pz, dd, G) && ok;
                const T sdl = sgn * o[3];
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    T su = 0, sv = 0;
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        su += us[a] * G[a][b];
                        sv += us[3 + a] * G[a][b];
                    }
                    o[5 + b] = sdl * su;
                    o[8 + b] = sdl * sv;
                }
            }
            if (!ok && !fail) fail = 1;
            if (henon) {
                const T fa = sel3<T>(hax, o[0], o[1], o[2]);
                // grazing test in cells per unit tau (physical velocity over the cell width)
                T fn = fa;
                if constexpr (RECT) fn = kF64 ? fa / sel3<T>(hax, dd[0], dd[1], dd[2]) : fa * sel3<T>(hax, dd[0], dd[1], dd[2]);
                const bool bad = !(fn * hsign >= graze);
                if (bad && !fail) fail = 2;
                if (kF64) {
                    const T den = bad ? (T)1 : fa;
#pragma unroll
                    for (int c = 0; c < NS; c++) o[c] = o[c] / den;
                } else {
                    const T inv = bad ? (T)0 : (T)1 / fa;
#pragma unroll
                    for (int c = 0; c < NS; c++) o[c] *= inv;
                }
            }
            // (the 3/8 rule's last stage is kept too when the tape holds the
            // stage derivatives: all four enter its solution)
            if (s < NST - 1 || (TAPE && SCH != 0)) {
                k0[s] = o[0];
                k1[s] = o[1];
                k2[s] = o[2];
            }
            if (s < NST - 1) {
                if constexpr (DEV != 0) {
#pragma unroll
                    for (int c = 0; c < 6; c++) kd[s][c] = o[5 + c];
                }
            }
            if constexpr (DEV != 0) {
#pragma unroll
                for (int c = 0; c < 6; c++) ad[c] += Tab<T, SCH>::b(s) * o[5 + c];
            }
            const T b = Tab<T, SCH>::b(s);
            a4[0] += b * o[0];
            a4[1] += b * o[1];
            a4[2] += b * o[2];
            if constexpr (SCH == 0) {
                const T e = kF64 ? Fehlberg<T>::b5(s) : Fehlberg<T>::e(s);
                a5[0] += e * o[0];
                a5[1] += e * o[1];
                a5[2] += e * o[2];
            }
            l4 += b * o[3];
            tw4 += b * o[4];
        }

        if (fail == 1) {
            finish_bad<T, SPLIT, RECT>(A, R, L, FQSL_LINE_NULL_B);
            active = false;
            continue;
        }
        if (!henon) {
            const T nx = L.x + hh * a4[0], ny = L.y + hh * a4[1], nz = L.z + hh * a4[2];
            // err > tol (FP64: err = |y5 - y4| with both solutions formed as
            // written; FP32: err^2 = h^2 |sum (b5 - b4) k|^2 accumulated in FP64
            // and compared with tol^2, the step factor (tol/err)^(1/4) =
            // (tol^2/err^2)^(1/8) in float)
            T hn = L.h;  // fixed-step scheme: every trial is accepted, the step is kept
            if constexpr (SCH == 0) {
                double err = 0.0;
                float rf = 0.f;
                bool over, pos;
                if (kF64) {
                    double d0 = (double)((L.x + hh * a5[0]) - nx), d1 = (double)((L.y + hh * a5[1]) - ny),
                           d2 = (double)((L.z + hh * a5[2]) - nz);
                    if constexpr (RECT) {
                        // in cells of the start cell
                        d0 = d0 / (double)dd[0];
                        d1 = d1 / (double)dd[1];
                        d2 = d2 / (double)dd[2];
                    }
                    err = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    over = err > L.tol;
                    pos = err > 0.0;
                } else if (ACC) {
                    double ex = (double)a5[0], ey = (double)a5[1], ez = (double)a5[2];
                    if constexpr (RECT) {
                        ex *= (double)dd[0];
                        ey *= (double)dd[1];
                        ez *= (double)dd[2];
                    }
                    err = (double)(hh * hh) * (ex * ex + ey * ey + ez * ez);  // err^2
                    over = err > L.tol;
                    pos = err > 0.0;
                    rf = __fdividef(L.tolf2, (float)err);
                } else {
                    T e5[3] = {a5[0], a5[1], a5[2]};
                    if constexpr (RECT) {
                        e5[0] *= dd[0];
                        e5[1] *= dd[1];
                        e5[2] *= dd[2];
                    }
                    const float e2 = (float)(hh * hh) * (float)(e5[0] * e5[0] + e5[1] * e5[1] + e5[2] * e5[2]);
                    over = e2 > L.tolf2;
                    pos = e2 > 0.f;
                    rf = __fdividef(L.tolf2, e2);
                }
                if (over) {
                    if (L.h > hmin) {
                        const T q = kF64 ? (T)root4(L.tol / err) : (T)sqrtf(root4(rf));
                        T hn = L.h * fmax((T)0.1, (T)0.9 * q);
                        L.h = hn < hmin ? hmin : hn;
                        continue;
                    }
                    L.st |= FQSL_LINE_STALL;
                }
                if (pos) {
                    const T q = kF64 ? (T)root4(L.tol / err) : (T)sqrtf(root4(rf));
                    hn = L.h * fmin((T)4, (T)0.9 * q);
                } else {
                    hn = (T)4 * L.h;
                }
                hn = hn < hmin ? hmin : (hn > hmax ? hmax : hn);
            }
            if (inside<T, RECT>(f, nx, ny, nz)) {
                if constexpr (TAPE) tape_step<T, SCH ? NST : NST - 1>(A.tape, L, hh, k0, k1, k2, nx, ny, nz);
                L.x = nx;
                L.y = ny;
                L.z = nz;
                if constexpr (DEV != 0) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        L.u[c] = L.u[c] + hh * ad[c];
                        L.v[c] = L.v[c] + hh * ad[3 + c];
                    }
                }
                acc_add<T, ACC>(L, hh * l4, hh * tw4);
                L.h = hn;
                continue;
            }
            // exit: the first face the chord crosses (ties: lower axis first)
            int best = -1;
            T tb = (T)INFINITY;
            const T cur[3] = {L.x, L.y, L.z}, nxt[3] = {nx, ny, nz};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const T lo = lo_of<T, RECT>(f, a), hi = hi_of<T, RECT>(f, a);
                T t;
                int fc;
                if (nxt[a] < lo) {
                    t = (lo - cur[a]) / (nxt[a] - cur[a]);
                    fc = 2 * a;
                } else if (nxt[a] > hi) {
                    t = (hi - cur[a]) / (nxt[a] - cur[a]);
                    fc = 2 * a + 1;
                } else {
                    continue;
                }
                if (t < tb) {
                    tb = t;
                    best = fc;
                }
            }
            L.ox = nx;
            L.oy = ny;
            L.oz = nz;
            if constexpr (DEV != 0) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    L.ou[c] = L.u[c] + hh * ad[c];
                    L.ov[c] = L.v[c] + hh * ad[3 + c];
                }
            }
            if (ACC) {
                L.ol = L.lacc + (double)(hh * l4);
                L.otw = L.twacc + (double)(hh * tw4);
            } else {
                L.ol = (double)(hh * l4);
                L.otw = (double)(hh * tw4);
            }
            L.t0 = tb;
            L.fc0 = best;
            L.hface = best;
            L.tries = 0;
            L.mode = 1;
            continue;
        }
        // exit step
        if (fail == 2) {
            L.mode = 0;
            if ((T)0.5 * L.h >= hmin) {
                L.h = (T)0.5 * L.h;
                continue;
            }
            // chord fallback onto the first crossed face
            T ex = L.x + L.t0 * (L.ox - L.x), ey = L.y + L.t0 * (L.oy - L.y), ez = L.z + L.t0 * (L.oz - L.z);
            const int a0 = L.fc0 >> 1;
            const T v0 = (L.fc0 & 1) ? hi_of<T, RECT>(f, a0) : lo_of<T, RECT>(f, a0);
            if (a0 == 0) ex = v0;
            else if (a0 == 1) ey = v0;
            else ez = v0;
            if (ACC) {
                L.lacc = L.lacc + (double)L.t0 * (L.ol - L.lacc);
                L.twacc = L.twacc + (double)L.t0 * (L.otw - L.twacc);
            } else {
                acc_add<T, ACC>(L, (T)((double)L.t0 * L.ol), (T)((double)L.t0 * L.otw));
            }
            L.st |= FQSL_LINE_CHORD;
            if constexpr (TAPE) tape_end(A.tape, L, kTapeChord + L.fc0, ex, ey, ez, L.h);
            T eu[3], ev[3];
            if constexpr (DEV != 0) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    eu[c] = L.u[c] + L.t0 * (L.ou[c] - L.u[c]);
                    ev[c] = L.v[c] + L.t0 * (L.ov[c] - L.v[c]);
                }
            }
            active = finish_dir<T, ACC, DEV, SPLIT, RECT>(A, R, L, ex, ey, ez, L.fc0, eu, ev);
            waiting = active && A0.p.sync_dirs;
            continue;
        }
        T tx = L.x + hh * a4[0], ty = L.y + hh * a4[1], tz = L.z + hh * a4[2];
        if (hax == 0) tx = target;
        else if (hax == 1) ty = target;
        else tz = target;
        int nf = -1;
        {
            const T tt[3] = {tx, ty, tz};
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (b == hax || nf >= 0) continue;
                if (tt[b] < lo_of<T, RECT>(f, b)) nf = 2 * b;
                else if (tt[b] > hi_of<T, RECT>(f, b)) nf = 2 * b + 1;
            }
        }
        if (nf >= 0 && L.tries < 2) {
            L.hface = nf;
            L.tries++;
            continue;
        }
        if (nf >= 0) {
            tx = fmin(fmax(tx, lo_of<T, RECT>(f, 0)), hi_of<T, RECT>(f, 0));
            ty = fmin(fmax(ty, lo_of<T, RECT>(f, 1)), hi_of<T, RECT>(f, 1));
            tz = fmin(fmax(tz, lo_of<T, RECT>(f, 2)), hi_of<T, RECT>(f, 2));
        }
        acc_add<T, ACC>(L, hh * l4, hh * tw4);
        if constexpr (TAPE) tape_end(A.tape, L, (nf >= 0 ? kTapeExitClamped : kTapeExit) + L.hface, tx, ty, tz, (T)0);
        T eu[3], ev[3];
        if constexpr (DEV != 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                eu[c] = L.u[c] + hh * ad[c];
                ev[c] = L.v[c] + hh * ad[3 + c];
            }
        }
        active = finish_dir<T, ACC, DEV, SPLIT, RECT>(A, R, L, tx, ty, tz, L.hface, eu, ev);
        waiting = active && A0.p.sync_dirs;
    }
}

// FP32 seed set-up for every lattice seed, one thread each (convergent): the
// index-space seed, Bn0, the S0 rotation decision and the per-line tolerance
// (Sec. 4, Eq. tol), or the final record of a seed outside the box or on a
// null field.
template <bool RECT = false>
__device__ __forceinline__ void seed_prep_f32(const TraceArgs &A, long long idx)
{
    const Lattice &G = A.lat;
    const FieldView &f = A.f;
    const LineRecs &R = A.rec;
    // 32-bit index arithmetic (a lattice holds fewer than 2^31 seeds)
    const unsigned u = (unsigned)idx, n1 = (unsigned)G.n1, n12 = (unsigned)(G.n1 * G.n2);
    const unsigned k = u / n12, rem = u - k * n12, j = rem / n1, i = rem - j * n1;
    const double fi = half_odd(i), fj = half_odd(j), fk = half_odd(k);
    double xi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) xi[a] = fma(fk, G.xa3[a], fma(fj, G.xa2[a], fma(fi, G.xa1[a], G.xo[a])));
    const float x = (float)xi[0], y = (float)xi[1], z = (float)xi[2];
    uint8_t fl = 0;
    unsigned bad = 0;
    double bn0 = 0.0, tol = ctl_perp(A.p);
    const bool in = in_box<float, RECT>(f, xi);
    if (!in) {
        bad = FQSL_LINE_OUTSIDE;
    } else {
        float B0[3], J0[3], rd[3];
        gatherg<RECT>(f, x, y, z, B0, J0, false);
        step_dd<float, RECT>(f, x, y, z, rd);
        const float b0 = B0[0] * rd[0], b1 = B0[1] * rd[1], b2 = B0[2] * rd[2];
        const float bb = b0 * b0 + b1 * b1 + b2 * b2;
        const float nB = sqrtf(B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2]);
        if (!(bb > 0.f) || !(bb < INFINITY) || !(nB > 0.f)) {
            bad = FQSL_LINE_NULL_B;
        } else {
            const float bn = B0[0] * (float)G.n0[0] + B0[1] * (float)G.n0[1] + B0[2] * (float)G.n0[2];
            if (bn < 0.f) fl |= kSeedNegS0;
            if (A.p.method == 2) {
                bn0 = f2d(nB);
            } else {
                const float ratio = fabsf(bn) / nB;
                bool on_face = false;
                if (G.normal_axis >= 0) {
                    const double xa = xi[G.normal_axis];
                    on_face = (xa == dlo<float, RECT>(f, G.normal_axis)) || (xa == dhi<float, RECT>(f, G.normal_axis));
                }
                if (G.allow_rot && ratio < (float)A.p.rot && !on_face) {
                    fl |= kSeedRotated;
                    bn0 = f2d(nB);
                    const unsigned slot = atomicAdd(A.q.rot_count, 1u);
                    A.q.rot_seed[slot] = (int32_t)idx;
                    A.q.rot_slot[idx] = (int32_t)slot + 1;
                } else if (A.p.scheme == 1) {
                    bn0 = f2d(bn);
                    tol = fmax(A.p.step * f2d(ratio), A.p.step_min);  // Eq. step
                } else {
                    bn0 = f2d(bn);
                    const float xr = fmaxf(ratio, (float)A.p.rot);
                    const float g = A.p.texp == 1.5 ? xr * sqrtf(xr) : __powf(xr, (float)A.p.texp);
                    tol = A.p.tol * f2d(g);
                }
            }
        }
    }
    R.bn0[idx] = bn0;
    if (A.prep.fu) {
        // Method II: S0 perpendicular to B, U0, V0 its frame (Sec. 4)
        float4 fu = make_float4(0.f, 0.f, 0.f, 0.f), fv = fu;
        if (!bad) {
            float B0[3], J0[3];
            gatherg<RECT>(f, x, y, z, B0, J0, false);
            const double b0 = B0[0], b1 = B0[1], b2 = B0[2];
            const double nB = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
            const double bh[3] = {b0 / nB, b1 / nB, b2 / nB};
            double u[3], v[3];
            perp_frame(bh, u, v);
            fu = make_float4((float)u[0], (float)u[1], (float)u[2], 0.f);
            fv = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
        }
        A.prep.fu[idx] = fu;
        A.prep.fv[idx] = fv;
    }
    if (bad) {
        fl |= kSeedDone;
        write_end32(R, idx, 0, x, y, z, -1);
        write_end32(R, idx, 1, x, y, z, -1);
        R.st[idx] = (uint8_t)bad;
        R.steps[idx] = 0;
    }
    // w: tol^2, or with the fixed-step scheme the line's step
    A.prep.seed[idx] = make_float4(x, y, z, A.p.scheme == 1 ? (float)tol : (float)(tol * tol));
    A.prep.flags[idx] = fl;
}

}  // namespace trace
}  // namespace fqsl
