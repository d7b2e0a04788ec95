// Device building blocks of the discrete adjoint (adjoint.cu): trilinear
// gathers with the interpolant's derivative and the adjoint scatter, the
// stage VJP and Jacobian of the line equation, and the kernels of the
// reverse sweep (passes A1, A2, B, C), templated on the stage scheme so that
// the RKF45 and fixed-step instantiations live in separate translation units.
#pragma once

#include <math.h>

#include "trace.cuh"

namespace fqsl {

namespace adj {

// The stages of one step's solution: RKF45's 4th-order solution (its sixth
// stage has zero weight there, so five) or Kutta's 3/8 rule (the fixed-step
// scheme, four).
template <typename T, int SCH>
struct Stages {
    static constexpr int N = SCH ? 4 : 5;
    static __device__ __forceinline__ T a(int s, int r) { return trace::Tab<T, SCH>::a(s, r); }
    static __device__ __forceinline__ T b(int s) { return trace::Tab<T, SCH>::b(s); }
};

// Failed index checks (the access is skipped and the first failure kept for
// the host): 1 chunk id, 2 steps in a chunk, 3 end code, 4 cell of a gather or
// scatter, 5 footpoint-adjoint index.
__device__ __forceinline__ void record_fail(unsigned long long *err, unsigned code, long long value)
{
    if (!err) return;
    const unsigned long long w = ((unsigned long long)code << 56) | ((unsigned long long)value & ((1ull << 56) - 1));
    atomicCAS(err, 0ull, w);
    atomicAdd(err + 1, 1ull);
}

// the 8 corners of the cell at node base lie in the cube (else record it)
__device__ __forceinline__ bool cell_ok(const FieldView &f, long long base)
{
    const bool ok = base >= 0 && base + (long long)f.nx * f.ny + f.nx + 1 < f.nodes;
    if (!ok) record_fail(f.err, 4, base);
    return ok;
}

// ---------------------------------------------------------------------------
// trilinear interpolation with the derivative of the interpolant
// ---------------------------------------------------------------------------
// Cell and fractions as the tracer's gather forms them: cell = floor(xi)
// clamped to [0, n-2]; weight of corner (m, q, p) = prod of (frac or 1-frac).
// On a stretched grid (Sec. 2.2) the cell is the one the tracer's search finds
// (a discrete choice, not differentiated) and the weights are Eq. w0's in
// physical coordinates, whose derivative along axis a is -+ 1/width_a.
template <typename T>
struct Cell {
    long long base;  // node of corner (0, 0, 0)
    T w0[3], w1[3];  // weights of the lower and upper corner along each axis
    T rw[3];         // stretched grid: 1 / width of the cell along each axis
};

__device__ __forceinline__ Cell<float> cell_of(const FieldView &f, float x, float y, float z)
{
    const float cx = fminf(fmaxf(floorf(x), 0.f), f.cmax[0]);
    const float cy = fminf(fmaxf(floorf(y), 0.f), f.cmax[1]);
    const float cz = fminf(fmaxf(floorf(z), 0.f), f.cmax[2]);
    Cell<float> c;
    c.base = ((long long)trace::small_int(cz) * f.ny + trace::small_int(cy)) * f.nx + trace::small_int(cx);
    c.w1[0] = x - cx;
    c.w1[1] = y - cy;
    c.w1[2] = z - cz;
    for (int a = 0; a < 3; a++) c.w0[a] = 1.f - c.w1[a];
    return c;
}

__device__ __forceinline__ Cell<double> cell_of(const FieldView &f, double x, double y, double z)
{
    const int cx = trace::cell_floor64(x, f.nx), cy = trace::cell_floor64(y, f.ny), cz = trace::cell_floor64(z, f.nz);
    Cell<double> c;
    c.base = ((long long)cz * f.ny + (long long)cy) * f.nx + (long long)cx;
    // the FP64 gather forms omega_0 = (c+1) - xi and omega_1 = 1 - omega_0
    c.w0[0] = trace::int_f64(cx + 1) - x;
    c.w0[1] = trace::int_f64(cy + 1) - y;
    c.w0[2] = trace::int_f64(cz + 1) - z;
    for (int a = 0; a < 3; a++) c.w1[a] = 1.0 - c.w0[a];
    return c;
}

// stretched grid, FP32: the forward's cell records {x_c, x_{c+1}, 1/width}
// relative to the first node; the lower corner's weight (x_{c+1} - x)/width
__device__ __forceinline__ Cell<float> cell_of_rect(const FieldView &f, float x, float y, float z)
{
    trace::RectCells<float> rc;
    trace::rect_cells(f, x, y, z, rc);
    Cell<float> c;
    c.base = ((long long)rc.c[2] * f.ny + rc.c[1]) * f.nx + rc.c[0];
    const float p[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        c.w0[a] = (rc.r[a].y - p[a]) * rc.r[a].z;
        c.w1[a] = 1.f - c.w0[a];
        c.rw[a] = rc.r[a].z;
    }
    return c;
}

// stretched grid, FP64: physical coordinates, Eqs. w0, w1 as the forward
// evaluates them
__device__ __forceinline__ Cell<double> cell_of_rect(const FieldView &f, double x, double y, double z)
{
    trace::RectCells<double> rc;
    trace::rect_cells(f, x, y, z, rc);
    Cell<double> c;
    c.base = ((long long)rc.c[2] * f.ny + rc.c[1]) * f.nx + rc.c[0];
    const double p[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double2 cr = rc.r[a];
        c.w0[a] = (cr.y - p[a]) / (cr.y - cr.x);
        c.w1[a] = 1.0 - c.w0[a];
        c.rw[a] = 1.0 / (cr.y - cr.x);
    }
    return c;
}

template <bool RECT, typename T>
__device__ __forceinline__ Cell<T> cellg(const FieldView &f, T x, T y, T z)
{
    if constexpr (RECT) return cell_of_rect(f, x, y, z);
    else return cell_of(f, x, y, z);
}

// The step's scale per axis, fixed at its start (the tracer's step_dd): FP64
// the spacing or, on a stretched grid, the widths of the start point's cell;
// FP32 their reciprocals.
template <bool RECT, typename T>
__device__ __forceinline__ void step_scale(const FieldView &f, T x, T y, T z, T dd[3])
{
    if constexpr (RECT) {
        trace::RectCells<T> rc;
        trace::rect_cells(f, x, y, z, rc);
        trace::dd_of(rc, dd);
    } else {
        trace::step_dd<T, false>(f, x, y, z, dd);
    }
}

// 1 / scale: bt_a = B_a rho_a
template <typename T>
__device__ __forceinline__ T rho_of(T dd)
{
    if constexpr (sizeof(T) == 8) return (T)1 / dd;
    else return dd;
}

__device__ __forceinline__ void load6(const FieldView &f, long long node, float v[6])
{
    trace::load_rec32((const char *)f.rec + (size_t)node * 32u, v[0], v[1], v[2], v[3], v[4], v[5]);
}

__device__ __forceinline__ void load6(const FieldView &f, long long node, double v[6])
{
    trace::load_node(f, node, v[0], v[1], v[2], v[3], v[4], v[5]);
}

// node of corner (m, q, p) and its weight and weight gradient (in state
// coordinates: index units, or physical on a stretched grid)
template <typename T, bool RECT = false>
__device__ __forceinline__ long long corner(const FieldView &f, const Cell<T> &c, int m, int q, int p, T &w, T dw[3])
{
    const T wx = m ? c.w1[0] : c.w0[0];
    const T wy = q ? c.w1[1] : c.w0[1];
    const T wz = p ? c.w1[2] : c.w0[2];
    w = wx * wy * wz;
    dw[0] = (m ? (T)1 : (T)-1) * wy * wz;
    dw[1] = (q ? (T)1 : (T)-1) * wx * wz;
    dw[2] = (p ? (T)1 : (T)-1) * wx * wy;
    if constexpr (RECT) {
        dw[0] *= c.rw[0];
        dw[1] *= c.rw[1];
        dw[2] *= c.rw[2];
    }
    return c.base + (long long)p * f.nx * f.ny + (long long)q * f.nx + m;
}

// V = (B, curl B) at the cell position and dV[a][c] = d V_c / d xi_a
template <typename T, bool RECT = false>
__device__ __forceinline__ void interp_d(const FieldView &f, const Cell<T> &c, T V[6], T dV[3][6])
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        V[k] = (T)0;
        dV[0][k] = dV[1][k] = dV[2][k] = (T)0;
    }
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) {
                T w, dw[3], v[6];
                const long long node = corner<T, RECT>(f, c, m, q, p, w, dw);
                load6(f, node, v);
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    V[k] += w * v[k];
                    dV[0][k] += dw[0] * v[k];
                    dV[1][k] += dw[1] * v[k];
                    dV[2][k] += dw[2] * v[k];
                }
            }
}

// scatter w * Vbar into the 6 adjoint slots of a node
__device__ __forceinline__ void scatter_node(float *acc, long long node, float w, const float Vb[6])
{
    float4 *p = (float4 *)(acc + 8 * node);
    atomicAdd(p, make_float4(w * Vb[0], w * Vb[1], w * Vb[2], w * Vb[3]));
    atomicAdd((float2 *)(p + 1), make_float2(w * Vb[4], w * Vb[5]));
}

__device__ __forceinline__ void scatter_node(double *acc, long long node, double w, const double Vb[6])
{
    double *p = acc + 8 * node;
#pragma unroll
    for (int k = 0; k < 6; k++) atomicAdd(p + k, w * Vb[k]);
}

template <typename T, typename AccT>
__device__ __forceinline__ void scatter(const FieldView &f, const Cell<T> &c, const T Vb[6], AccT *acc)
{
    if (Vb[0] == (T)0 && Vb[1] == (T)0 && Vb[2] == (T)0 && Vb[3] == (T)0 && Vb[4] == (T)0 && Vb[5] == (T)0) return;
    AccT vb[6];
#pragma unroll
    for (int k = 0; k < 6; k++) vb[k] = (AccT)Vb[k];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) {
                T w, dw[3];
                const long long node = corner(f, c, m, q, p, w, dw);
                scatter_node(acc, node, (AccT)w, vb);
            }
}

// ---------------------------------------------------------------------------
// stage VJP: the line equation's right-hand side at position p,
//   F = sgn bt/|bt| (bt_a = B_a / d_a), dtw = (J.B)/(4 pi B^2) |B|/|bt|,
// given the adjoints of F and dtw (bars(F, dtw, Fb, dtwb) forms them from the
// stage's own values): scatters the adjoints of B, J into the node grid and
// returns the adjoint of p.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T inv_spacing(const FieldView &f, int a);
template <>
__device__ __forceinline__ float inv_spacing<float>(const FieldView &f, int a)
{
    return f.rd[a];
}
template <>
__device__ __forceinline__ double inv_spacing<double>(const FieldView &f, int a)
{
    return 1.0 / f.d[a];
}

template <typename T>
struct V3 {
    T x, y, z;
};

// Stage VJP. ax < 0: the adjoints of F and dtw are
// (kb, twb); ax >= 0 (exit step): kb and twb are the adjoints of K = F/F_ax
// and dtw/F_ax, converted with the stage's own F_ax. All-zero adjoints
// return at once. RECT (stretched grid, Sec. 2.3): F = sgn B/|bt| with bt_a =
// B_a/D_a, D (dd) the widths of the step's start cell, held fixed.
template <typename T, typename AccT, bool RECT = false>
__device__ __forceinline__ V3<T> stage_vjp(const FieldView &f, const T dd[3], T sgn, T px, T py, T pz, int ax, T kb0,
                                           T kb1, T kb2, T twb, AccT *acc)
{
    V3<T> r = {(T)0, (T)0, (T)0};
    if (kb0 == (T)0 && kb1 == (T)0 && kb2 == (T)0 && twb == (T)0) return r;
    const Cell<T> c = cellg<RECT>(f, px, py, pz);
    if (!cell_ok(f, c.base)) return r;
    T V[6], dV[3][6];
    interp_d<T, RECT>(f, c, V, dV);
    if constexpr (RECT) {
        const T rho[3] = {rho_of(dd[0]), rho_of(dd[1]), rho_of(dd[2])};
        const T bt[3] = {V[0] * rho[0], V[1] * rho[1], V[2] * rho[2]};
        const T bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
        const T BB = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
        const T nbt = sqrt(bb), m = sqrt(BB);
        const T c4 = (T)12.566370614359172 * m * nbt;  // 4 pi |B| |bt|
        const T JB = V[3] * V[0] + V[4] * V[1] + V[5] * V[2];
        const T dtw = JB / c4;
        const T F[3] = {sgn * V[0] / nbt, sgn * V[1] / nbt, sgn * V[2] / nbt};
        T Fb[3] = {kb0, kb1, kb2}, dtwb = twb;
        if (ax >= 0) {
            const T fa = F[ax];
            const T g = (kb0 * F[0] + kb1 * F[1] + kb2 * F[2] + twb * dtw) / (fa * fa);
            Fb[0] = kb0 / fa;
            Fb[1] = kb1 / fa;
            Fb[2] = kb2 / fa;
            Fb[ax] -= g;
            dtwb = twb / fa;
        }
        // F_a = sgn B_a / |bt|: Bbar_j = sgn (Fbar_j / |bt| - (Fbar . B) rho_j^2 B_j / |bt|^3)
        const T FB = Fb[0] * V[0] + Fb[1] * V[1] + Fb[2] * V[2];
        T Vb[6];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const T r2 = rho[a] * rho[a] * V[a];
            Vb[a] = sgn * (Fb[a] / nbt - FB * r2 / (nbt * bb)) + dtwb * (V[3 + a] / c4 - dtw * V[a] / BB - dtw * r2 / bb);
            Vb[3 + a] = dtwb * V[a] / c4;
        }
        T pb[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            T sacc = (T)0;
#pragma unroll
            for (int k = 0; k < 6; k++) sacc += dV[a][k] * Vb[k];
            pb[a] = sacc;
        }
        scatter(f, c, Vb, acc);
        r.x = pb[0];
        r.y = pb[1];
        r.z = pb[2];
        return r;
    }
    const T rd[3] = {inv_spacing<T>(f, 0), inv_spacing<T>(f, 1), inv_spacing<T>(f, 2)};
    const T bt[3] = {V[0] * rd[0], V[1] * rd[1], V[2] * rd[2]};
    const T bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
    const T BB = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const T nbt = sqrt(bb), m = sqrt(BB);
    const T u[3] = {bt[0] / nbt, bt[1] / nbt, bt[2] / nbt};
    const T c4 = (T)12.566370614359172 * m * nbt;  // 4 pi |B| |bt|
    const T JB = V[3] * V[0] + V[4] * V[1] + V[5] * V[2];
    const T dtw = JB / c4;
    T Fb[3] = {kb0, kb1, kb2}, dtwb = twb;
    if (ax >= 0) {
        // K = F / F_ax and twK = dtw / F_ax
        const T F[3] = {sgn * u[0], sgn * u[1], sgn * u[2]};
        const T fa = F[ax];
        const T g = (kb0 * F[0] + kb1 * F[1] + kb2 * F[2] + twb * dtw) / (fa * fa);
        Fb[0] = kb0 / fa;
        Fb[1] = kb1 / fa;
        Fb[2] = kb2 / fa;
        Fb[ax] -= g;
        dtwb = twb / fa;
    }
    // F = sgn bt/|bt|: d(bt/|bt|) = (I - u u^T)/|bt|
    const T uf = u[0] * Fb[0] + u[1] * Fb[1] + u[2] * Fb[2];
    T Vb[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const T btb = sgn * (Fb[a] - u[a] * uf) / nbt;
        Vb[a] = btb * rd[a] + dtwb * (V[3 + a] / c4 - dtw * V[a] / BB - dtw * u[a] * rd[a] / nbt);
        Vb[3 + a] = dtwb * V[a] / c4;
    }
    T pb[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T s = (T)0;
#pragma unroll
        for (int k = 0; k < 6; k++) s += dV[a][k] * Vb[k];
        pb[a] = s;
    }
    scatter(f, c, Vb, acc);
    r.x = pb[0];
    r.y = pb[1];
    r.z = pb[2];
    return r;
}

template <typename T>
struct Rhs {
    T F[3], dl, dtw;
};

// right-hand side in the tracer's own form (the same function the forward
// ran; dd: the step's scale from step_scale, used on a stretched grid)
template <bool RECT = false>
__device__ __forceinline__ Rhs<float> rhs_fwd(const FieldView &f, const float dd[3], float sgn, float x, float y,
                                              float z)
{
    float o[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if constexpr (RECT) trace::rhs_rect(f, dd, sgn, x, y, z, o);
    else if (cell_ok(f, cell_of(f, x, y, z).base)) trace::rhs(f, f.rd, sgn, x, y, z, o);
    return Rhs<float>{{o[0], o[1], o[2]}, o[3], o[4]};
}

template <bool RECT = false>
__device__ __forceinline__ Rhs<double> rhs_fwd(const FieldView &f, const double dd[3], double sgn, double x, double y,
                                               double z)
{
    double o[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if constexpr (RECT) trace::rhs_rect(f, dd, sgn, x, y, z, o);
    else if (cell_ok(f, cell_of(f, x, y, z).base)) trace::rhs(f, f.d, sgn, x, y, z, o);
    return Rhs<double>{{o[0], o[1], o[2]}, o[3], o[4]};
}

// One step of the 4th-order solution from x, as the tracer forms it: RKF45
// (SCH 0; stages 0..4, the 4th-order weights of stages 1 and 5 are zero) or
// the 3/8 rule (SCH 1; stages 0..3). ax < 0: an
// accepted step of size h; ax >= 0: the exit step, whose independent variable
// is the ax index coordinate (h = target - x_ax, RHS divided by its ax
// component). Writes the end state and, per stage, the (divided) derivative
// and Tw integrand k[s] = {F (3), dtw}.
template <typename T, int SCH, bool RECT = false>
__device__ __forceinline__ void advance(const FieldView &f, const T dd[3], T sgn, const T x[3], T h, int ax, T x4[3],
                                        T k[5][4])
{
    constexpr bool kF64 = sizeof(T) == 8;
    T a4[3] = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < Stages<T, SCH>::N; s++) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Stages<T, SCH>::a(s, r);
            px += c * k[r][0];
            py += c * k[r][1];
            pz += c * k[r][2];
        }
        const Rhs<T> o = rhs_fwd<RECT>(f, dd, sgn, x[0] + h * px, x[1] + h * py, x[2] + h * pz);
        T F[4] = {o.F[0], o.F[1], o.F[2], o.dtw};
        if (ax >= 0) {
            const T fa = o.F[ax];
            if (kF64) {
#pragma unroll
                for (int a = 0; a < 4; a++) F[a] = F[a] / fa;
            } else {
                const T inv = (T)1 / fa;
#pragma unroll
                for (int a = 0; a < 4; a++) F[a] = F[a] * inv;
            }
        }
#pragma unroll
        for (int a = 0; a < 4; a++) k[s][a] = F[a];
        const T b = Stages<T, SCH>::b(s);
        a4[0] += b * F[0];
        a4[1] += b * F[1];
        a4[2] += b * F[2];
    }
    x4[0] = x[0] + h * a4[0];
    x4[1] = x[1] + h * a4[1];
    x4[2] = x[2] + h * a4[2];
}

// Reverse of that step (its stages are evaluated again here: cheaper than
// keeping them per step): on entry xb is the adjoint of the end state and wb
// that of the Tw increment; on exit xb is the adjoint of x through the stages
// and, for the exit step (ax >= 0), *db the adjoint of its length h.
template <typename T, typename AccT, int SCH, bool RECT = false>
__device__ __forceinline__ void step_reverse(const FieldView &f, T sgn, const T x[3], T h, int ax, T xb[3], T wb,
                                             T *db, AccT *acc)
{
    T k[5][4], x4[3], dd[3];
    step_scale<RECT>(f, x[0], x[1], x[2], dd);
    advance<T, SCH, RECT>(f, dd, sgn, x, h, ax, x4, k);
    T kb[5][3];
    T d = 0;
#pragma unroll
    for (int s = 0; s < Stages<T, SCH>::N; s++) {
        const T b = Stages<T, SCH>::b(s);
#pragma unroll
        for (int a = 0; a < 3; a++) kb[s][a] = h * b * xb[a];
        d += b * (k[s][0] * xb[0] + k[s][1] * xb[1] + k[s][2] * xb[2] + k[s][3] * wb);
    }
    T xin[3] = {xb[0], xb[1], xb[2]};
#pragma unroll
    for (int s = Stages<T, SCH>::N - 1; s >= 0; s--) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Stages<T, SCH>::a(s, r);
            px += c * k[r][0];
            py += c * k[r][1];
            pz += c * k[r][2];
        }
        const V3<T> pb = stage_vjp<T, AccT, RECT>(f, dd, sgn, x[0] + h * px, x[1] + h * py, x[2] + h * pz, ax,
                                                  kb[s][0], kb[s][1], kb[s][2], h * Stages<T, SCH>::b(s) * wb, acc);
        xin[0] += pb.x;
        xin[1] += pb.y;
        xin[2] += pb.z;
        d += pb.x * px + pb.y * py + pb.z * pz;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = h * Stages<T, SCH>::a(s, r);
            kb[r][0] += c * pb.x;
            kb[r][1] += c * pb.y;
            kb[r][2] += c * pb.z;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) xb[a] = xin[a];
    if (db) *db = d;
}

// ---------------------------------------------------------------------------
// The reverse sweep, parallel in time. The adjoint of one accepted step is
// linear in the adjoints of its end state and of the Tw sum:
//   xbar_i = J_i^T xbar_{i+1} + g_i wbar,
// J_i = d x_{i+1} / d x_i, g_i = d (Tw increment) / d x_i. So, rather than one
// thread walking a whole direction backwards (a chain of ~15 dependent field
// gathers per step), three passes:
//   A1 (per tape chunk) recompute the chunk's states and stage derivatives
//                       from its checkpoint;
//   A2 (per step)       each step's J_i, g_i by forward-mode tangents;
//   B (per half-line)   the exit step's VJP (with its scatter), then the
//                       recurrence above over the stored J_i, g_i (no gathers),
//                       storing each step's xbar_{i+1};
//   C (per step)        each step's stage VJPs and scatters given xbar_{i+1}.
// Only A1 walks a chunk (at most k steps) sequentially, so the longest chain of
// dependent gathers is one chunk's recompute instead of a whole line's reverse.
// ---------------------------------------------------------------------------

// V, dV/dxi at p and, from them, F, dtw and their position Jacobians:
// Jm[i][j] = dF_i/dp_j, g[j] = d dtw/dp_j. Returns false (values zero) when the
// cell check fails.
template <typename T, bool RECT = false>
__device__ __forceinline__ bool stage_jac(const FieldView &f, const T dd[3], T sgn, T px, T py, T pz, T F[3], T &dtw,
                                          T Jm[3][3], T g[3])
{
    const Cell<T> c = cellg<RECT>(f, px, py, pz);
    if (!cell_ok(f, c.base)) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            F[i] = g[i] = (T)0;
            Jm[i][0] = Jm[i][1] = Jm[i][2] = (T)0;
        }
        dtw = (T)0;
        return false;
    }
    T V[6], dV[3][6];
    interp_d<T, RECT>(f, c, V, dV);
    if constexpr (RECT) {
        // F = sgn B/|bt|, bt_a = B_a rho_a (rho = 1/D of the step's start cell):
        // dF_i/dp_j = sgn (dB_i/dp_j - B_i q_j / |bt|^2) / |bt|, q_j = sum_b rho_b^2 B_b dB_b/dp_j
        const T rho[3] = {rho_of(dd[0]), rho_of(dd[1]), rho_of(dd[2])};
        const T bt[3] = {V[0] * rho[0], V[1] * rho[1], V[2] * rho[2]};
        const T bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
        const T BB = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
        const T nbt = sqrt(bb), m = sqrt(BB);
        const T c4 = (T)12.566370614359172 * m * nbt;
        const T JB = V[3] * V[0] + V[4] * V[1] + V[5] * V[2];
        dtw = JB / c4;
        T dB[3], dJ[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            F[a] = sgn * V[a] / nbt;
            dB[a] = V[3 + a] / c4 - dtw * V[a] / BB - dtw * rho[a] * rho[a] * V[a] / bb;
            dJ[a] = V[a] / c4;
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const T q = rho[0] * rho[0] * V[0] * dV[j][0] + rho[1] * rho[1] * V[1] * dV[j][1] +
                        rho[2] * rho[2] * V[2] * dV[j][2];
#pragma unroll
            for (int i = 0; i < 3; i++) Jm[i][j] = sgn * (dV[j][i] - V[i] * q / bb) / nbt;
            g[j] = dB[0] * dV[j][0] + dB[1] * dV[j][1] + dB[2] * dV[j][2] + dJ[0] * dV[j][3] + dJ[1] * dV[j][4] +
                   dJ[2] * dV[j][5];
        }
        return true;
    }
    const T rd[3] = {inv_spacing<T>(f, 0), inv_spacing<T>(f, 1), inv_spacing<T>(f, 2)};
    const T bt[3] = {V[0] * rd[0], V[1] * rd[1], V[2] * rd[2]};
    const T bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
    const T BB = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const T nbt = sqrt(bb), m = sqrt(BB);
    const T u[3] = {bt[0] / nbt, bt[1] / nbt, bt[2] / nbt};
    const T c4 = (T)12.566370614359172 * m * nbt;  // 4 pi |B| |bt|
    const T JB = V[3] * V[0] + V[4] * V[1] + V[5] * V[2];
    dtw = JB / c4;
    // d dtw / dB and d dtw / dJ
    T dB[3], dJ[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        F[a] = sgn * u[a];
        dB[a] = V[3 + a] / c4 - dtw * V[a] / BB - dtw * u[a] * rd[a] / nbt;
        dJ[a] = V[a] / c4;
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        // F = sgn u(bt), u = bt/|bt|: dF_i/dp_j = sgn (rd_i dB_i/dp_j - u_i q_j)/|bt|
        const T q = u[0] * rd[0] * dV[j][0] + u[1] * rd[1] * dV[j][1] + u[2] * rd[2] * dV[j][2];
#pragma unroll
        for (int i = 0; i < 3; i++) Jm[i][j] = sgn * (rd[i] * dV[j][i] - u[i] * q) / nbt;
        g[j] = dB[0] * dV[j][0] + dB[1] * dV[j][1] + dB[2] * dV[j][2] + dJ[0] * dV[j][3] + dJ[1] * dV[j][4] +
               dJ[2] * dV[j][5];
    }
    return true;
}

// Reverse of an accepted step whose stage derivatives k are known (from
// pass A1): xb in = adjoint of the end state, out = adjoint of x.
template <typename T, typename AccT, int SCH, bool RECT = false>
__device__ __forceinline__ void step_reverse_k(const FieldView &f, T sgn, const T x[3], T h, const T k[5][3], T xb[3],
                                               T wb, AccT *acc)
{
    T kb[5][3], dd[3];
    step_scale<RECT>(f, x[0], x[1], x[2], dd);
#pragma unroll
    for (int s = 0; s < Stages<T, SCH>::N; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) kb[s][a] = h * Stages<T, SCH>::b(s) * xb[a];
#pragma unroll
    for (int s = Stages<T, SCH>::N - 1; s >= 0; s--) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Stages<T, SCH>::a(s, r);
            px += c * k[r][0];
            py += c * k[r][1];
            pz += c * k[r][2];
        }
        const V3<T> pb = stage_vjp<T, AccT, RECT>(f, dd, sgn, x[0] + h * px, x[1] + h * py, x[2] + h * pz, -1,
                                                  kb[s][0], kb[s][1], kb[s][2], h * Stages<T, SCH>::b(s) * wb, acc);
        xb[0] += pb.x;
        xb[1] += pb.y;
        xb[2] += pb.z;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = h * Stages<T, SCH>::a(s, r);
            kb[r][0] += c * pb.x;
            kb[r][1] += c * pb.y;
            kb[r][2] += c * pb.z;
        }
    }
}

constexpr int kMaxChunk = 32;  // largest steps per tape chunk

// Half-lines of the taped map: 2 line + end for the lattice lines, then
// 2 n + 2 (4 slot + q) + end for the extra lines of rotated seeds.
__device__ __forceinline__ long long halves_of(const AdjArgs &A)
{
    if (!A.rot_count) return 2 * A.n;
    const long long r = (long long)*A.rot_count;
    return 2 * A.n + 8 * (r < A.n ? r : A.n);
}

// status of the line that half-line hl belongs to
__device__ __forceinline__ unsigned half_status(const AdjArgs &A, long long hl)
{
    return hl < 2 * A.n ? A.rec.st[hl >> 1] : A.ext.st[(hl - 2 * A.n) >> 1];
}

// Does half-line hl carry a nonzero adjoint (footpoint or Tw weight)? Extra
// lines carry no Tw weight.
__device__ __forceinline__ bool half_live(const AdjArgs &A, long long hl, double &w)
{
    w = (A.dTw && hl < 2 * A.n) ? A.dTw[hl >> 1] : 0.0;
    if (!(w == w) || fabs(w) == INFINITY) w = 0.0;
    const double *xb = A.xbar + 3 * hl;
    return w != 0.0 || xb[0] != 0.0 || xb[1] != 0.0 || xb[2] != 0.0;
}

// The chunk's half-line, orientation and step count; false if nothing to do.
__device__ __forceinline__ bool chunk_of(const AdjArgs &A, long long c, long long &hl, int &n, int &sgn, double &w)
{
    const Tape &tp = A.tape;
    hl = tp.owner[c];
    if (hl < 0 || hl >= halves_of(A)) {
        record_fail(A.f.err, 1, c);
        return false;
    }
    if (half_status(A, hl) & kBad) return false;
    if (!half_live(A, hl, w)) return false;
    const int4 hd = tp.head[hl];
    if (hd.x < 0 || hd.z < 0) return false;
    n = hd.x == (int)c ? hd.y : tp.k;
    if (n < 0 || n > tp.k || n > kMaxChunk) {
        record_fail(A.f.err, 2, n);
        return false;
    }
    sgn = hd.w;
    return true;
}

// A kept state and a step's stage derivatives (the layouts of Tape::wx, wk)
// in 16-byte read-only loads.
__device__ __forceinline__ void load_state(const float *p, float x[3])
{
    const float4 q = __ldg((const float4 *)p);
    x[0] = q.x;
    x[1] = q.y;
    x[2] = q.z;
}
__device__ __forceinline__ void load_state(const double *p, double x[3])
{
    const double2 a = __ldg((const double2 *)p), b = __ldg((const double2 *)p + 1);
    x[0] = a.x;
    x[1] = a.y;
    x[2] = b.x;
}
template <typename T, int NS>
__device__ __forceinline__ void load_stages(const T *p, T k[5][3])
{
    constexpr int N = (3 * NS + 3) / 4 * 4;  // values to load: the stages, rounded up to whole float4
    T v[kStageStride];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < N; q += 4) {
            const float4 a = __ldg((const float4 *)(p + q));
            v[q] = a.x;
            v[q + 1] = a.y;
            v[q + 2] = a.z;
            v[q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; q += 2) {
            const double2 a = __ldg((const double2 *)(p + q));
            v[q] = a.x;
            v[q + 1] = a.y;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) k[s][a] = v[3 * s + a];
}

// pass A1: the states and stage derivatives of every chunk, from its
// checkpoint (the only sequential recompute), unless the forward kept them
// (AdjArgs::stored); either way the list of live steps
template <typename T, typename TT, int SCH, bool RECT = false>
__global__ void __launch_bounds__(128) k_adj_states(const AdjArgs A)
{
    const Tape &tp = A.tape;
    const int K = tp.k;
    T *WX = (T *)A.wx;
    T *WK = (T *)A.wk;
    const TT *X = (const TT *)tp.xi;
    const TT *H = (const TT *)tp.h;
    const int lane = threadIdx.x & 31;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < A.chunks;
         c += (long long)gridDim.x * blockDim.x) {
        long long hl;
        int n = 0, sg = 0;
        double w;
        const bool live = chunk_of(A, c, hl, n, sg, w);
        A.cinfo[c] = live ? make_int4(n, sg, (int)hl, 1) : make_int4(0, 0, -1, 0);
        // this chunk's steps in the compacted list of passes A2 and C: one
        // atomic per warp. The lanes still in the loop are a prefix of the
        // warp (consecutive c); the *_sync intrinsics below converge them.
        const long long left = A.chunks - (c - lane);
        const unsigned mask = left >= 32 ? 0xffffffffu : ((1u << (unsigned)left) - 1u);
        const int v = live ? n : 0;
        int inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(mask, inc, d);
            if (lane >= d) inc += t;
        }
        const int last = 31 - __clz(mask);
        const int total = __shfl_sync(mask, inc, last);
        unsigned long long base = 0;
        if (lane == 0 && total > 0) base = atomicAdd(A.nsteps, (unsigned long long)total);
        base = __shfl_sync(mask, base, 0) + (unsigned long long)(inc - v);
        if (!live) continue;
        for (int i = 0; i < n; i++) A.steps[base + i] = (int32_t)(c * K + i);
        if (A.stored) continue;  // the forward kept the states and stage derivatives
        T x[3] = {(T)X[4 * c], (T)X[4 * c + 1], (T)X[4 * c + 2]};
        T *wx = WX + c * (K + 1) * kStateStride;
        T *wk = WK + c * K * kStageStride;
        trace::store_state(wx, x[0], x[1], x[2]);
        for (int i = 0; i < n; i++) {
            T x4[3], kt[5][4], dd[3];
            step_scale<RECT>(A.f, x[0], x[1], x[2], dd);
            advance<T, SCH, RECT>(A.f, dd, (T)sg, x, (T)H[c * K + i], -1, x4, kt);
            T v[kStageStride];
#pragma unroll
            for (int q = 0; q < kStageStride; q++) v[q] = (T)0;
#pragma unroll
            for (int s = 0; s < Stages<T, SCH>::N; s++)
#pragma unroll
                for (int a = 0; a < 3; a++) v[3 * s + a] = kt[s][a];
            trace::store_vec<T, kStageStride>(wk + kStageStride * i, v);
#pragma unroll
            for (int a = 0; a < 3; a++) x[a] = x4[a];
            trace::store_state(wx + kStateStride * (i + 1), x[0], x[1], x[2]);
        }
    }
}

// entry t of the compacted step list: the step's flat index j = c k + i,
// its chunk c and index i, the half-line's orientation and Tw weight
__device__ __forceinline__ bool step_of(const AdjArgs &A, long long t, long long &j, long long &c, int &i, int &sg,
                                        double &w)
{
    const int K = A.tape.k;
    j = A.steps[t];
    c = j / K;
    i = (int)(j - c * K);
    if (j < 0 || c >= A.chunks) {
        record_fail(A.f.err, 1, j);
        return false;
    }
    const int4 ci = A.cinfo[c];
    if (!ci.w || i >= ci.x) return false;
    sg = ci.y;
    w = (A.dTw && ci.z < 2 * A.n) ? A.dTw[ci.z >> 1] : 0.0;
    if (!(w == w) || fabs(w) == INFINITY) w = 0.0;
    return true;
}

// pass A2: each step's Jacobian J^T and Tw gradient (one thread per step)
template <typename T, typename TT, int SCH, bool RECT = false>
__global__ void __launch_bounds__(128) k_adj_jac(const AdjArgs A)
{
    const int K = A.tape.k;
    const T *WX = (const T *)A.wx;
    const T *WK = (const T *)A.wk;
    T *WJ = (T *)A.wj;
    const TT *H = (const TT *)A.tape.h;
    const long long steps = (long long)*A.nsteps;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < steps;
         t += (long long)gridDim.x * blockDim.x) {
        long long j, c;
        int i, sg;
        double w;
        if (!step_of(A, t, j, c, i, sg, w)) continue;
        T x[3], k[5][3];
        load_state(WX + (c * (K + 1) + i) * kStateStride, x);
        load_stages<T, Stages<T, SCH>::N>(WK + j * kStageStride, k);
        const T h = (T)H[j];
        const T sgn = (T)sg;
        // the step's scale, fixed at its start (stretched grid: its start cell)
        T dd[3];
        step_scale<RECT>(A.f, x[0], x[1], x[2], dd);
        // tangents: P_s = d p_s / d x = I + h sum_r a_sr D_r, D_s = dF(p_s)/dp P_s
        T D[5][3][3], Ds[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gs[3] = {0, 0, 0};
#pragma unroll
        for (int s = 0; s < Stages<T, SCH>::N; s++) {
            T px = 0, py = 0, pz = 0;
            T P[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
            for (int r = 0; r < s; r++) {
                const T cc = Stages<T, SCH>::a(s, r);
                px += cc * k[r][0];
                py += cc * k[r][1];
                pz += cc * k[r][2];
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) P[a][b] += h * cc * D[r][a][b];
            }
            T F[3], dtw, Jm[3][3], g[3];
            stage_jac<T, RECT>(A.f, dd, sgn, x[0] + h * px, x[1] + h * py, x[2] + h * pz, F, dtw, Jm, g);
            const T b4 = Stages<T, SCH>::b(s);
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    D[s][a][b] = Jm[a][0] * P[0][b] + Jm[a][1] * P[1][b] + Jm[a][2] * P[2][b];
                    Ds[a][b] += b4 * D[s][a][b];
                }
#pragma unroll
            for (int b = 0; b < 3; b++) gs[b] += b4 * (g[0] * P[0][b] + g[1] * P[1][b] + g[2] * P[2][b]);
        }
        T *wj = WJ + j * 12;
#pragma unroll
        for (int a = 0; a < 3; a++) {
#pragma unroll
            for (int b = 0; b < 3; b++) wj[3 * a + b] = (a == b ? (T)1 : (T)0) + h * Ds[b][a];
            wj[9 + a] = h * gs[a];
        }
    }
}

// pass B: per half-line, the exit step's VJP and the recurrence over its
// steps; an extra line's half-line also keeps the adjoint of its seed
// One step of pass B's recurrence: store the step's end-state adjoint y, then
// y <- J^T y + g wbar (J = {J^T row-major (9), g (3)}).
// The 12 values of a step's pass-A2 record (16-byte aligned: records are 48 or
// 96 bytes from an aligned base) in 16-byte read-only loads.
template <typename T>
__device__ __forceinline__ void load_jrec(const T *p, T J[12])
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int v = 0; v < 3; v++) {
            const float4 q = __ldg((const float4 *)p + v);
            J[4 * v + 0] = q.x;
            J[4 * v + 1] = q.y;
            J[4 * v + 2] = q.z;
            J[4 * v + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int v = 0; v < 6; v++) {
            const double2 q = __ldg((const double2 *)p + v);
            J[2 * v + 0] = q.x;
            J[2 * v + 1] = q.y;
        }
    }
}

template <typename T>
__device__ __forceinline__ void adj_rec_step(const T J[12], T wb, T y[3], T *out)
{
    out[0] = y[0];
    out[1] = y[1];
    out[2] = y[2];
    const T z0 = J[0] * y[0] + J[1] * y[1] + J[2] * y[2] + J[9] * wb;
    const T z1 = J[3] * y[0] + J[4] * y[1] + J[5] * y[2] + J[10] * wb;
    const T z2 = J[6] * y[0] + J[7] * y[1] + J[8] * y[2] + J[11] * wb;
    y[0] = z0;
    y[1] = z1;
    y[2] = z2;
}

template <typename T, typename AccT, typename TT, int SCH, bool RECT = false>
__global__ void __launch_bounds__(128) k_adj_lines(const AdjArgs A)
{
    const Tape &tp = A.tape;
    const FieldView &f = A.f;
    const int K = tp.k;
    const T *WX = (const T *)A.wx;
    const T *WJ = (const T *)A.wj;
    T *WB = (T *)A.wb;
    AccT *acc = (AccT *)A.acc;
    const long long halves = halves_of(A);
    for (long long hl = blockIdx.x * (long long)blockDim.x + threadIdx.x; hl < halves;
         hl += (long long)gridDim.x * blockDim.x) {
        if (half_status(A, hl) & kBad) continue;
        double w;
        if (!half_live(A, hl, w)) continue;
        const int4 hd = tp.head[hl];
        if (hd.x < 0 || hd.z < 0) continue;
        if (hd.x >= A.chunks) {
            record_fail(f.err, 1, hd.x);
            continue;
        }
        const int code = hd.z;
        const bool chord = code >= kTapeChord && code < kTapeChord + 6;
        const bool clamped = code >= kTapeExitClamped && code < kTapeExitClamped + 6;
        if (!(chord || clamped || (code >= kTapeExit && code < kTapeExit + 6))) {
            record_fail(f.err, 3, code);
            continue;
        }
        if (hd.y < 0 || hd.y > K) {
            record_fail(f.err, 2, hd.y);
            continue;
        }
        const T wb = (T)w;
        const T sgn = (T)hd.w;
        const int face = code - (chord ? kTapeChord : (clamped ? kTapeExitClamped : kTapeExit));
        const int fax = face >> 1;
        // the face in state coordinates (physical on a stretched grid)
        const T target = (face & 1) ? trace::hi_of<T, RECT>(f, fax) : trace::lo_of<T, RECT>(f, fax);
        T xb[3];
#pragma unroll
        for (int a = 0; a < 3; a++) xb[a] = (T)A.xbar[3 * hl + a];
        // the exiting step from the state after the last accepted step
        T x[3];
        load_state(WX + ((long long)hd.x * (K + 1) + hd.y) * kStateStride, x);
        T h, d = 0, ws = wb;
        int ax = -1;
        T yb[3] = {xb[0], xb[1], xb[2]}, keep[3] = {0, 0, 0}, y[3];
        T x4[3], kt[5][4];
        bool zero = false;  // a zero-length exit step
        if (chord) {
            // end = x + t0 (x4 - x), t0 = (target - x_ax)/(x4_ax - x_ax); Tw gains t0 of the step's increment
            h = (T)((const TT *)tp.xe)[4 * hl + 3];
            T dd[3];
            step_scale<RECT>(f, x[0], x[1], x[2], dd);
            advance<T, SCH, RECT>(f, dd, sgn, x, h, -1, x4, kt);
            T dtw = 0;
#pragma unroll
            for (int s = 0; s < Stages<T, SCH>::N; s++) dtw += Stages<T, SCH>::b(s) * kt[s][3];
            dtw *= h;
            const T den = x4[fax] - x[fax];
            const T t0 = (target - x[fax]) / den;
            T cb[3] = {xb[0], xb[1], xb[2]};
            cb[fax] = (T)0;
            const T t0b = cb[0] * (x4[0] - x[0]) + cb[1] * (x4[1] - x[1]) + cb[2] * (x4[2] - x[2]) + wb * dtw;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                yb[a] = t0 * cb[a];
                keep[a] = ((T)1 - t0) * cb[a];
            }
            yb[fax] -= t0b * t0 / den;
            keep[fax] += t0b * (t0 - (T)1) / den;
            ws = t0 * wb;
        } else {
            // exit step onto the face: its ax coordinate is the face, the
            // others are clamped into the box when the code says so
            ax = fax;
            h = target - x[fax];
            yb[fax] = (T)0;
            if (h == (T)0) {
                // a zero-length exit step (a seed on the face): the end is x,
                // all stages sit at x, nothing is scattered; only the length's
                // dependence on x_ax remains: d = K(x) . yb + twK(x) wbar
                // no earlier step: a lattice seed's adjoint is not needed
                if (hd.y == 0 && tp.prev[hd.x] < 0 && hl < 2 * A.n) continue;
                T dd[3];
                step_scale<RECT>(f, x[0], x[1], x[2], dd);
                const Rhs<T> o = rhs_fwd<RECT>(f, dd, sgn, x[0], x[1], x[2]);
                const T fa = o.F[fax];
                d = (o.F[0] * yb[0] + o.F[1] * yb[1] + o.F[2] * yb[2] + o.dtw * wb) / fa;
                y[0] = yb[0];
                y[1] = yb[1];
                y[2] = yb[2];
                y[fax] -= d;
                zero = true;
            } else if (clamped) {
                T dd[3];
                step_scale<RECT>(f, x[0], x[1], x[2], dd);
                advance<T, SCH, RECT>(f, dd, sgn, x, h, ax, x4, kt);
#pragma unroll
                for (int b = 0; b < 3; b++)
                    if (b != fax && (x4[b] < trace::lo_of<T, RECT>(f, b) || x4[b] > trace::hi_of<T, RECT>(f, b)))
                        yb[b] = (T)0;
            }
        }
        if (!zero) {
            step_reverse<T, AccT, SCH, RECT>(f, sgn, x, h, ax, yb, ws, ax >= 0 ? &d : (T *)nullptr, acc);
#pragma unroll
            for (int a = 0; a < 3; a++) y[a] = yb[a] + keep[a];
            if (ax >= 0) y[fax] -= d;  // h = target - x_ax
        }
        // the accepted steps, last first: store each step's end-state adjoint,
        // then xbar_i = J_i^T xbar_{i+1} + g_i wbar
        // (the Jacobians were written by pass A2 and are read-only here: their
        // loads go ahead of the chain, four steps at a time)
        int c = hd.x, n = hd.y;
        for (;;) {
            const T *__restrict__ wj = WJ + (long long)c * K * 12;
            T *__restrict__ wbp = WB + (long long)c * K * 3;
            const int pc = tp.prev[c];
            int i = n - 1;
            for (; i >= 3; i -= 4) {
                T Jb[4][12];
#pragma unroll
                for (int u = 0; u < 4; u++) load_jrec(wj + 12 * (i - u), Jb[u]);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    adj_rec_step(Jb[u], wb, y, wbp + 3 * (i - u));
                }
            }
            for (; i >= 0; i--) {
                T Jr[12];
                load_jrec(wj + 12 * i, Jr);
                adj_rec_step(Jr, wb, y, wbp + 3 * i);
            }
            if (pc < 0 || pc >= c) break;  // chunks of a half-line are taken in increasing order
            c = pc;
            n = K;
        }
        if (hl >= 2 * A.n) {
            double *xs = A.xseed + 3 * (hl - 2 * A.n);
            xs[0] = (double)y[0];
            xs[1] = (double)y[1];
            xs[2] = (double)y[2];
        }
    }
}

// pass C: the stage VJPs of every step, given its end-state adjoint (one
// thread per step)
template <typename T, typename AccT, typename TT, int SCH, bool RECT = false>
__global__ void __launch_bounds__(128) k_adj_rev(const AdjArgs A)
{
    const int K = A.tape.k;
    const T *WX = (const T *)A.wx;
    const T *WB = (const T *)A.wb;
    const T *WK = (const T *)A.wk;
    const TT *H = (const TT *)A.tape.h;
    AccT *acc = (AccT *)A.acc;
    const long long steps = (long long)*A.nsteps;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < steps;
         t += (long long)gridDim.x * blockDim.x) {
        long long j, c;
        int i, sg;
        double w;
        if (!step_of(A, t, j, c, i, sg, w)) continue;
        T yb[3] = {WB[3 * j], WB[3 * j + 1], WB[3 * j + 2]};
        T x[3], ks[5][3];
        load_state(WX + (c * (K + 1) + i) * kStateStride, x);
        load_stages<T, Stages<T, SCH>::N>(WK + j * kStageStride, ks);
        step_reverse_k<T, AccT, SCH, RECT>(A.f, (T)sg, x, (T)H[j], ks, yb, (T)w, acc);
    }
}

// ---------------------------------------------------------------------------
// host side: grid sizes and the passes
// ---------------------------------------------------------------------------
inline int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

inline unsigned grid_for(long long n, int per_block, int cap_per_sm)
{
    long long b = (n + per_block - 1) / per_block;
    const long long cap = (long long)sm_count() * cap_per_sm;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// the reverse sweep's passes A1, A2, B, C of a taped map traced with stage scheme SCH
template <typename T, typename AccT, typename TT, int SCH, bool RECT = false>
void reverse_passes(const AdjArgs &a, cudaStream_t s)
{
    const unsigned gc = grid_for(a.chunks, 128, 16);
    const unsigned gs = grid_for(a.chunks * a.tape.k, 128, 16);
    const unsigned gl = grid_for(2 * a.n, 128, 16);
    k_adj_states<T, TT, SCH, RECT><<<gc, 128, 0, s>>>(a);
    k_adj_jac<T, TT, SCH, RECT><<<gs, 128, 0, s>>>(a);
    k_adj_lines<T, AccT, TT, SCH, RECT><<<gl, 128, 0, s>>>(a);
    k_adj_rev<T, AccT, TT, SCH, RECT><<<gs, 128, 0, s>>>(a);
}

}  // namespace adj

}  // namespace fqsl
