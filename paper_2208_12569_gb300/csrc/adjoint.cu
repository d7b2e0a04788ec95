// Discrete adjoint of the plane-lattice Q and Tw maps (Method I): d/dB of
// sum_s dQ[s] Q[s] + dTw[s] Tw[s] for given per-seed weights (the paper has no
// derivative; this is the reverse mode of the traced computation).
//
// The forward pass (the lattice tracer with TAPE set) records, per direction
// of every line, its accepted step sizes in chunks of k steps with the state
// at each chunk's first step, and how the direction ended. The derivative is
// that of the computation with those step sizes, exit faces and exit kinds
// frozen; every position, stage value, exit-step length, chord parameter and
// field value varies with B. Kernels, in launch order:
//   q_vjp        per seed: the VJP of Method I's Q (Eqs. D+-2, D+-3, Q+- with
//                |det D| -> |Bn1/Bn2|, Eq. Bn1) onto the footpoints of the
//                lines its differences used, and of Bn at the seed and at
//                both ends onto B (trilinear weights, Sec. 2.2);
//   reverse      per half-line (warps take 8x4-seed tiles of one end from a
//                work counter): walk the chunks backwards; recompute each
//                chunk's states from its checkpoint, then reverse the exit
//                step (Henon step or chord) and every RKF45 step (4th-order
//                solution, stages in reverse), scattering the adjoints of the
//                interpolated B and curl B into a node grid;
//   curl_adjoint per node: dB += dB_interp + curl^T dJ_interp (the transpose
//                of the curl grid's stencils, Eq. tw).
// The state is recomputed in the traced precision T; the node grid
// accumulates in AccT (float with vector atomics, or double).
#include <math.h>

#include "trace.cuh"

namespace fqsl {

namespace adj {

using trace::Fehlberg;

// ---------------------------------------------------------------------------
// trilinear interpolation with the derivative of the interpolant
// ---------------------------------------------------------------------------
// Cell and fractions as the tracer's gather forms them: cell = floor(xi)
// clamped to [0, n-2]; weight of corner (m, q, p) = prod of (frac or 1-frac).
template <typename T>
struct Cell {
    long long base;  // node of corner (0, 0, 0)
    T w0[3], w1[3];  // weights of the lower and upper corner along each axis
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
    const double cx = trace::clampcell<double>(floor(x), f.nx);
    const double cy = trace::clampcell<double>(floor(y), f.ny);
    const double cz = trace::clampcell<double>(floor(z), f.nz);
    Cell<double> c;
    c.base = ((long long)cz * f.ny + (long long)cy) * f.nx + (long long)cx;
    // the FP64 gather forms omega_0 = (c+1) - xi and omega_1 = 1 - omega_0
    c.w0[0] = (cx + 1.0) - x;
    c.w0[1] = (cy + 1.0) - y;
    c.w0[2] = (cz + 1.0) - z;
    for (int a = 0; a < 3; a++) c.w1[a] = 1.0 - c.w0[a];
    return c;
}

__device__ __forceinline__ void load6(const FieldView &f, long long node, float v[6])
{
    trace::load_rec32((const char *)f.rec + (size_t)node * 32u, v[0], v[1], v[2], v[3], v[4], v[5]);
}

__device__ __forceinline__ void load6(const FieldView &f, long long node, double v[6])
{
    trace::load_node(f, node, v[0], v[1], v[2], v[3], v[4], v[5]);
}

// node of corner (m, q, p) and its weight and weight gradient
template <typename T>
__device__ __forceinline__ long long corner(const FieldView &f, const Cell<T> &c, int m, int q, int p, T &w, T dw[3])
{
    const T wx = m ? c.w1[0] : c.w0[0];
    const T wy = q ? c.w1[1] : c.w0[1];
    const T wz = p ? c.w1[2] : c.w0[2];
    w = wx * wy * wz;
    dw[0] = (m ? (T)1 : (T)-1) * wy * wz;
    dw[1] = (q ? (T)1 : (T)-1) * wx * wz;
    dw[2] = (p ? (T)1 : (T)-1) * wx * wy;
    return c.base + (long long)p * f.nx * f.ny + (long long)q * f.nx + m;
}

// V = (B, curl B) at the cell position and dV[a][c] = d V_c / d xi_a
template <typename T>
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
                const long long node = corner(f, c, m, q, p, w, dw);
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

template <typename T, typename AccT, typename Bars>
__device__ __forceinline__ void stage_vjp(const FieldView &f, T sgn, T px, T py, T pz, Bars bars, T pb[3], AccT *acc)
{
    const Cell<T> c = cell_of(f, px, py, pz);
    T V[6], dV[3][6];
    interp_d(f, c, V, dV);
    const T rd[3] = {inv_spacing<T>(f, 0), inv_spacing<T>(f, 1), inv_spacing<T>(f, 2)};
    const T bt[3] = {V[0] * rd[0], V[1] * rd[1], V[2] * rd[2]};
    const T bb = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
    const T BB = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const T nbt = sqrt(bb), m = sqrt(BB);
    const T u[3] = {bt[0] / nbt, bt[1] / nbt, bt[2] / nbt};
    const T F[3] = {sgn * u[0], sgn * u[1], sgn * u[2]};
    const T c4 = (T)12.566370614359172 * m * nbt;  // 4 pi |B| |bt|
    const T JB = V[3] * V[0] + V[4] * V[1] + V[5] * V[2];
    const T dtw = JB / c4;
    T Fb[3], dtwb;
    bars(F, dtw, Fb, dtwb);
    // F: d(bt/|bt|) = (I - u u^T)/|bt|
    const T uf = u[0] * Fb[0] + u[1] * Fb[1] + u[2] * Fb[2];
    T Vb[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const T btb = sgn * (Fb[a] - u[a] * uf) / nbt;
        Vb[a] = btb * rd[a] + dtwb * (V[3 + a] / c4 - dtw * V[a] / BB - dtw * u[a] * rd[a] / nbt);
        Vb[3 + a] = dtwb * V[a] / c4;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T s = (T)0;
#pragma unroll
        for (int k = 0; k < 6; k++) s += dV[a][k] * Vb[k];
        pb[a] = s;
    }
    scatter(f, c, Vb, acc);
}

// right-hand side in the tracer's own form (the same function the forward ran)
__device__ __forceinline__ void rhs_fwd(const FieldView &f, float sgn, float x, float y, float z, float o[5])
{
    o[0] = o[1] = o[2] = o[3] = o[4] = 0.f;
    trace::rhs(f, f.rd, sgn, x, y, z, o);
}

__device__ __forceinline__ void rhs_fwd(const FieldView &f, double sgn, double x, double y, double z, double o[5])
{
    o[0] = o[1] = o[2] = o[3] = o[4] = 0.0;
    trace::rhs(f, f.d, sgn, x, y, z, o);
}

// one accepted step of the 4th-order solution, as the tracer forms it (stages
// 0..4: the 4th-order weights of stages 1 and 5 are zero); also the stage
// derivatives k and the Tw increment
template <typename T>
__device__ __forceinline__ void advance(const FieldView &f, T sgn, const T x[3], T h, T x4[3], T k[5][3], T *dtw4)
{
    T a4[3] = {0, 0, 0}, tw4 = 0;
#pragma unroll
    for (int s = 0; s < 5; s++) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Fehlberg<T>::a(s, r);
            px += c * k[r][0];
            py += c * k[r][1];
            pz += c * k[r][2];
        }
        T o[5];
        rhs_fwd(f, sgn, x[0] + h * px, x[1] + h * py, x[2] + h * pz, o);
        k[s][0] = o[0];
        k[s][1] = o[1];
        k[s][2] = o[2];
        const T b = Fehlberg<T>::b4(s);
        a4[0] += b * o[0];
        a4[1] += b * o[1];
        a4[2] += b * o[2];
        tw4 += b * o[4];
    }
    x4[0] = x[0] + h * a4[0];
    x4[1] = x[1] + h * a4[1];
    x4[2] = x[2] + h * a4[2];
    if (dtw4) *dtw4 = h * tw4;
}

// Reverse of one accepted step of size h from x: on entry xb is the adjoint of
// the step's end state and wb that of its Tw increment; on exit xb is the
// adjoint of x.
template <typename T, typename AccT>
__device__ __forceinline__ void step_reverse(const FieldView &f, T sgn, const T x[3], T h, T xb[3], T wb, AccT *acc)
{
    T k[5][3], x4[3];
    advance(f, sgn, x, h, x4, k, (T *)nullptr);
    T kb[5][3];
#pragma unroll
    for (int s = 0; s < 5; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) kb[s][a] = h * Fehlberg<T>::b4(s) * xb[a];
    T xin[3] = {xb[0], xb[1], xb[2]};
#pragma unroll
    for (int s = 4; s >= 0; s--) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Fehlberg<T>::a(s, r);
            px += c * k[r][0];
            py += c * k[r][1];
            pz += c * k[r][2];
        }
        const T twb = h * Fehlberg<T>::b4(s) * wb;
        T pb[3];
        stage_vjp<T, AccT>(
            f, sgn, x[0] + h * px, x[1] + h * py, x[2] + h * pz,
            [&](const T *, T, T *Fb, T &dtwb) {
                Fb[0] = kb[s][0];
                Fb[1] = kb[s][1];
                Fb[2] = kb[s][2];
                dtwb = twb;
            },
            pb, acc);
#pragma unroll
        for (int a = 0; a < 3; a++) xin[a] += pb[a];
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = h * Fehlberg<T>::a(s, r);
#pragma unroll
            for (int a = 0; a < 3; a++) kb[r][a] += c * pb[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) xb[a] = xin[a];
}

// Reverse of the exit step from x onto face `face` (the face-normal index
// coordinate is the independent variable, Sec. 2.1): the end point is
// x + delta sum b4 K_s, K = F/F_ax, delta = target - x_ax, with its ax
// coordinate set to the face and (clamped) the others clamped into the box.
template <typename T, typename AccT>
__device__ __forceinline__ void exit_reverse(const FieldView &f, T sgn, const T x[3], int face, bool clamped, T xb[3],
                                             T wb, AccT *acc)
{
    constexpr bool kF64 = sizeof(T) == 8;
    const int ax = face >> 1;
    const int nax = ax == 0 ? f.nx : (ax == 1 ? f.ny : f.nz);
    const T target = (face & 1) ? (T)(nax - 1) : (T)0;
    const T delta = target - x[ax];
    T K[5][3], twK[5];
    T a4[3] = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < 5; s++) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Fehlberg<T>::a(s, r);
            px += c * K[r][0];
            py += c * K[r][1];
            pz += c * K[r][2];
        }
        T o[5];
        rhs_fwd(f, sgn, x[0] + delta * px, x[1] + delta * py, x[2] + delta * pz, o);
        const T fa = trace::sel3<T>(ax, o[0], o[1], o[2]);
        if (kF64) {
#pragma unroll
            for (int a = 0; a < 3; a++) K[s][a] = o[a] / fa;
            twK[s] = o[4] / fa;
        } else {
            const T inv = (T)1 / fa;
#pragma unroll
            for (int a = 0; a < 3; a++) K[s][a] = o[a] * inv;
            twK[s] = o[4] * inv;
        }
        const T b = Fehlberg<T>::b4(s);
        a4[0] += b * K[s][0];
        a4[1] += b * K[s][1];
        a4[2] += b * K[s][2];
    }
    T eb[3] = {xb[0], xb[1], xb[2]};
    eb[ax] = (T)0;
    if (clamped) {
        const int nn[3] = {f.nx, f.ny, f.nz};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const T e = x[b] + delta * a4[b];
            if (b != ax && (e < (T)0 || e > (T)(nn[b] - 1))) eb[b] = (T)0;
        }
    }
    T db = 0;
    T Kb[5][3], twKb[5];
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const T b = Fehlberg<T>::b4(s);
        db += b * (K[s][0] * eb[0] + K[s][1] * eb[1] + K[s][2] * eb[2] + twK[s] * wb);
#pragma unroll
        for (int a = 0; a < 3; a++) Kb[s][a] = delta * b * eb[a];
        twKb[s] = delta * b * wb;
    }
    T xin[3] = {eb[0], eb[1], eb[2]};
#pragma unroll
    for (int s = 4; s >= 0; s--) {
        T px = 0, py = 0, pz = 0;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = Fehlberg<T>::a(s, r);
            px += c * K[r][0];
            py += c * K[r][1];
            pz += c * K[r][2];
        }
        T pb[3];
        stage_vjp<T, AccT>(
            f, sgn, x[0] + delta * px, x[1] + delta * py, x[2] + delta * pz,
            [&](const T *F, T dtw, T *Fb, T &dtwb) {
                // K = F / F_ax and twK = dtw / F_ax
                const T fa = F[ax];
                const T g = (Kb[s][0] * F[0] + Kb[s][1] * F[1] + Kb[s][2] * F[2] + twKb[s] * dtw) / (fa * fa);
                Fb[0] = Kb[s][0] / fa;
                Fb[1] = Kb[s][1] / fa;
                Fb[2] = Kb[s][2] / fa;
                Fb[ax] -= g;
                dtwb = twKb[s] / fa;
            },
            pb, acc);
#pragma unroll
        for (int a = 0; a < 3; a++) xin[a] += pb[a];
        db += pb[0] * px + pb[1] * py + pb[2] * pz;
#pragma unroll
        for (int r = 0; r < s; r++) {
            const T c = delta * Fehlberg<T>::a(s, r);
#pragma unroll
            for (int a = 0; a < 3; a++) Kb[r][a] += c * pb[a];
        }
    }
    xin[ax] -= db;
#pragma unroll
    for (int a = 0; a < 3; a++) xb[a] = xin[a];
}

// Reverse of the chord end: after an exiting step of size h from x to x4, the
// end is x + t0 (x4 - x) with t0 = (target - x_ax)/(x4_ax - x_ax), its ax
// coordinate set to the face; Tw gains t0 times the step's increment.
template <typename T, typename AccT>
__device__ __forceinline__ void chord_reverse(const FieldView &f, T sgn, const T x[3], int face, T h, T xb[3], T wb,
                                              AccT *acc)
{
    const int ax = face >> 1;
    const int nax = ax == 0 ? f.nx : (ax == 1 ? f.ny : f.nz);
    const T target = (face & 1) ? (T)(nax - 1) : (T)0;
    T k[5][3], x4[3], dtw;
    advance(f, sgn, x, h, x4, k, &dtw);
    const T den = x4[ax] - x[ax];
    const T t0 = (target - x[ax]) / den;
    T cb[3] = {xb[0], xb[1], xb[2]};
    cb[ax] = (T)0;
    const T t0b = cb[0] * (x4[0] - x[0]) + cb[1] * (x4[1] - x[1]) + cb[2] * (x4[2] - x[2]) + wb * dtw;
    T x4b[3] = {t0 * cb[0], t0 * cb[1], t0 * cb[2]};
    x4b[ax] -= t0b * t0 / den;
    T xin[3] = {((T)1 - t0) * cb[0], ((T)1 - t0) * cb[1], ((T)1 - t0) * cb[2]};
    xin[ax] += t0b * (t0 - (T)1) / den;
    step_reverse<T, AccT>(f, sgn, x, h, x4b, t0 * wb, acc);
#pragma unroll
    for (int a = 0; a < 3; a++) xb[a] = xin[a] + x4b[a];
}

constexpr int kMaxChunk = 64;  // largest steps per tape chunk

// Reverse sweep of half-line hl = 2 line + e (TT: the tape's scalar type).
template <typename T, typename AccT, typename TT>
__device__ __forceinline__ void reverse_half_line(const AdjArgs &A, long long line, int e, T (*xs)[3])
{
    const Tape &tp = A.tape;
    const long long hl = 2 * line + e;
    const int4 hd = tp.head[hl];
    if (hd.x < 0 || hd.z < 0) return;
    T xb[3];
#pragma unroll
    for (int a = 0; a < 3; a++) xb[a] = (T)A.xbar[3 * hl + a];
    double w = A.dTw ? A.dTw[line] : 0.0;
    if (!(w == w) || fabs(w) == INFINITY) w = 0.0;
    const T wb = (T)w;
    if (xb[0] == (T)0 && xb[1] == (T)0 && xb[2] == (T)0 && wb == (T)0) return;
    AccT *acc = (AccT *)A.acc;
    const FieldView &f = A.f;
    const T sgn = (T)hd.w;
    const TT *H = (const TT *)tp.h;
    const TT *X = (const TT *)tp.xi;
    // last chunk: its states up to the exit step
    int c = hd.x;
    int n = hd.y;
    xs[0][0] = (T)X[4 * (long long)c];
    xs[0][1] = (T)X[4 * (long long)c + 1];
    xs[0][2] = (T)X[4 * (long long)c + 2];
    for (int i = 0; i < n; i++) {
        T k[5][3];
        advance(f, sgn, xs[i], (T)H[(long long)c * tp.k + i], xs[i + 1], k, (T *)nullptr);
    }
    const int code = hd.z;
    if (code >= kTapeChord) {
        const T hx = (T)((const TT *)tp.xe)[4 * hl + 3];
        chord_reverse<T, AccT>(f, sgn, xs[n], code - kTapeChord, hx, xb, wb, acc);
    } else if (code >= kTapeExitClamped) {
        exit_reverse<T, AccT>(f, sgn, xs[n], code - kTapeExitClamped, true, xb, wb, acc);
    } else {
        exit_reverse<T, AccT>(f, sgn, xs[n], code - kTapeExit, false, xb, wb, acc);
    }
    for (;;) {
        for (int i = n - 1; i >= 0; i--)
            step_reverse<T, AccT>(f, sgn, xs[i], (T)H[(long long)c * tp.k + i], xb, wb, acc);
        const int pc = tp.prev[c];
        if (pc < 0 || pc >= c) break;  // chunks of a half-line are taken in increasing order
        c = pc;
        n = tp.k;
        xs[0][0] = (T)X[4 * (long long)c];
        xs[0][1] = (T)X[4 * (long long)c + 1];
        xs[0][2] = (T)X[4 * (long long)c + 2];
        for (int i = 0; i + 1 < n; i++) {
            T k[5][3];
            advance(f, sgn, xs[i], (T)H[(long long)c * tp.k + i], xs[i + 1], k, (T *)nullptr);
        }
    }
}

template <typename T, typename AccT, typename TT>
__global__ void __launch_bounds__(128) k_reverse(const AdjArgs A)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const Lattice &G = A.lat;
    const long long units = G.tiles_u * G.tiles_v * 2;  // (tile, end) pairs
    T xs[kMaxChunk + 1][3];
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(A.head, 1ull);
        u = __shfl_sync(FULL, u, 0);
        if ((long long)u >= units) break;
        const long long t = (long long)(u >> 1);
        const int e = (int)(u & 1);
        const long long i = (t % G.tiles_u) * kTileU + (lane % kTileU);
        const long long j = (t / G.tiles_u) * kTileV + (lane / kTileU);
        if (i < G.n1 && j < G.n2) {
            const long long line = i + G.n1 * j;
            if (!(A.rec.st[line] & kBad)) reverse_half_line<T, AccT, TT>(A, line, e, xs);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// VJP of Method I's Q and of Bn at the seed and at the ends (per seed)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void face_axes(int face, int &r0, int &r1)
{
    const int a = face >> 1;
    r0 = (a == 0) ? 1 : 0;
    r1 = (a == 2) ? 1 : 2;
}

// B_ax at index position p (traced precision), its gradient in index
// coordinates, and the scatter of bnb * e_ax onto the nodes
template <typename T, typename AccT>
__device__ __forceinline__ double bn_vjp(const FieldView &f, const T p[3], int ax, double bnb, double g[3], AccT *acc)
{
    const Cell<T> c = cell_of(f, p[0], p[1], p[2]);
    T V[6], dV[3][6];
    interp_d(f, c, V, dV);
    g[0] = (double)dV[0][ax];
    g[1] = (double)dV[1][ax];
    g[2] = (double)dV[2][ax];
    if (bnb != 0.0) {
        T Vb[6] = {0, 0, 0, 0, 0, 0};
        Vb[ax] = (T)bnb;
        scatter(f, c, Vb, acc);
    }
    return (double)V[ax];
}

template <typename T, typename AccT, typename TT>
__global__ void __launch_bounds__(128) k_q_vjp(const AdjArgs A)
{
    const Lattice &G = A.lat;
    const FieldView &f = A.f;
    const LineRecs &R = A.rec;
    const TT *XE = (const TT *)A.tape.xe;
    AccT *acc = (AccT *)A.acc;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
         idx += (long long)gridDim.x * blockDim.x) {
        const unsigned st = R.st[idx];
        if (st & (kBad | FQSL_LINE_ROTATED)) continue;
        const double qb = A.dQ ? A.dQ[idx] : 0.0;
        if (!(qb == qb) || qb == 0.0 || fabs(qb) == INFINITY) continue;
        const long long i = idx % G.n1, j = idx / G.n1;
        const long long ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
        long long nid[4];
        bool has[4];
        for (int q = 0; q < 4; q++) {
            has[q] = ni[q] >= 0 && ni[q] < G.n1 && nj[q] >= 0 && nj[q] < G.n2;
            nid[q] = has[q] ? ni[q] + G.n1 * nj[q] : 0;
        }
        const double inv[2] = {1.0 / G.du, 1.0 / G.dv};
        const int fe2[2] = {R.f1[idx], R.f2[idx]};
        // J_e[r][s] = sum over two lines of cf * xi_{ra[r]}(line, e)
        double Jm[2][2][2];
        long long ln[2][2][2];  // [e][s][plus/minus line]
        double cf[2][2][2];     // the two coefficients (index units; times d below)
        bool mixed = false;
        for (int e = 0; e < 2 && !mixed; e++) {
            int ra[2];
            face_axes(fe2[e], ra[0], ra[1]);
            for (int s = 0; s < 2 && !mixed; s++) {
                const int P = 2 * s, M = 2 * s + 1;
                const bool okp = has[P] && !(R.st[nid[P]] & kBad) && (e == 0 ? R.f1 : R.f2)[nid[P]] == fe2[e];
                const bool okm = has[M] && !(R.st[nid[M]] & kBad) && (e == 0 ? R.f1 : R.f2)[nid[M]] == fe2[e];
                if (okp && okm) {
                    ln[e][s][0] = nid[P];
                    ln[e][s][1] = nid[M];
                    cf[e][s][0] = 0.5 * inv[s];
                    cf[e][s][1] = -0.5 * inv[s];
                } else if (okp) {
                    ln[e][s][0] = nid[P];
                    ln[e][s][1] = idx;
                    cf[e][s][0] = inv[s];
                    cf[e][s][1] = -inv[s];
                } else if (okm) {
                    ln[e][s][0] = idx;
                    ln[e][s][1] = nid[M];
                    cf[e][s][0] = inv[s];
                    cf[e][s][1] = -inv[s];
                } else {
                    mixed = true;
                    break;
                }
                for (int r = 0; r < 2; r++) {
                    const int a = ra[r];
                    const double xp = (double)XE[4 * (2 * ln[e][s][0] + e) + a];
                    const double xm = (double)XE[4 * (2 * ln[e][s][1] + e) + a];
                    Jm[e][r][s] = (cf[e][s][0] * xp + cf[e][s][1] * xm) * f.d[a];
                }
            }
        }
        if (mixed) continue;
        // Q = |J2 adj(J1)|^2 |Bn1 Bn2| / Bn0^2
        const double Ad[2][2] = {{Jm[0][1][1], -Jm[0][0][1]}, {-Jm[0][1][0], Jm[0][0][0]}};
        double M[2][2], N = 0.0;
        for (int r = 0; r < 2; r++)
            for (int s = 0; s < 2; s++) {
                M[r][s] = Jm[1][r][0] * Ad[0][s] + Jm[1][r][1] * Ad[1][s];
                N += M[r][s] * M[r][s];
            }
        T pe[2][3];
        for (int e = 0; e < 2; e++)
            for (int a = 0; a < 3; a++) pe[e][a] = (T)XE[4 * (2 * idx + e) + a];
        double g1[3], g2[3];
        const int ax1 = fe2[0] >> 1, ax2 = fe2[1] >> 1;
        const double bn1 = bn_vjp<T, AccT>(f, pe[0], ax1, 0.0, g1, acc);
        const double bn2 = bn_vjp<T, AccT>(f, pe[1], ax2, 0.0, g2, acc);
        const double bn0 = R.bn0[idx];
        const double sc = fabs(bn1 * bn2) / (bn0 * bn0);
        const double Nb = qb * sc, sb = qb * N;
        // d N / d M = 2 M; M = J2 Ad
        double J2b[2][2], Adb[2][2];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 2; k++) {
                J2b[r][k] = 2.0 * Nb * (M[r][0] * Ad[k][0] + M[r][1] * Ad[k][1]);
                Adb[r][k] = 2.0 * Nb * (Jm[1][0][r] * M[0][k] + Jm[1][1][r] * M[1][k]);
            }
        double Jb[2][2][2];
        Jb[0][0][0] = Adb[1][1];
        Jb[0][0][1] = -Adb[0][1];
        Jb[0][1][0] = -Adb[1][0];
        Jb[0][1][1] = Adb[0][0];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 2; k++) Jb[1][r][k] = J2b[r][k];
        for (int e = 0; e < 2; e++) {
            int ra[2];
            face_axes(fe2[e], ra[0], ra[1]);
            for (int s = 0; s < 2; s++)
                for (int r = 0; r < 2; r++) {
                    const int a = ra[r];
                    const double v = Jb[e][r][s] * f.d[a];
                    atomicAdd(A.xbar + 3 * (2 * ln[e][s][0] + e) + a, cf[e][s][0] * v);
                    atomicAdd(A.xbar + 3 * (2 * ln[e][s][1] + e) + a, cf[e][s][1] * v);
                }
        }
        // |Bn1 Bn2| / Bn0^2
        const double sg1 = bn1 < 0.0 ? -1.0 : 1.0, sg2 = bn2 < 0.0 ? -1.0 : 1.0;
        const double bn1b = sb * sg1 * fabs(bn2) / (bn0 * bn0);
        const double bn2b = sb * sg2 * fabs(bn1) / (bn0 * bn0);
        const double bn0b = -2.0 * sb * fabs(bn1 * bn2) / (bn0 * bn0 * bn0);
        bn_vjp<T, AccT>(f, pe[0], ax1, bn1b, g1, acc);
        bn_vjp<T, AccT>(f, pe[1], ax2, bn2b, g2, acc);
        for (int a = 0; a < 3; a++) {
            atomicAdd(A.xbar + 3 * (2 * idx + 0) + a, bn1b * g1[a]);
            atomicAdd(A.xbar + 3 * (2 * idx + 1) + a, bn2b * g2[a]);
        }
        // Bn0 = B(seed) . n0
        T p0[3];
        if (A.prep.seed) {
            // the FP32 tracer's seed (its pre-pass)
            const float4 sd = A.prep.seed[idx];
            p0[0] = (T)sd.x;
            p0[1] = (T)sd.y;
            p0[2] = (T)sd.z;
        } else {
            // the FP64 tracer's seed: (r0 - o)/d as written
            double r0[3];
            trace::lattice_seed(G, i, j, 0, r0);
            for (int a = 0; a < 3; a++) p0[a] = (T)((r0[a] - f.o[a]) / f.d[a]);
        }
        const Cell<T> c0 = cell_of(f, p0[0], p0[1], p0[2]);
        const T Vb[6] = {(T)(bn0b * G.n0[0]), (T)(bn0b * G.n0[1]), (T)(bn0b * G.n0[2]), 0, 0, 0};
        scatter(f, c0, Vb, acc);
    }
}

// ---------------------------------------------------------------------------
// dB += dB_interp + curl^T dJ_interp (per node)
// ---------------------------------------------------------------------------
// coefficient of node jn in row i of the curl grid's derivative stencil along
// an axis of n nodes and spacing h
__device__ __forceinline__ double stencil(long long i, long long jn, long long n, double h)
{
    if (n == 2) return jn == 1 ? 1.0 / h : -1.0 / h;
    if (i == 0) return jn == 0 ? -1.5 / h : (jn == 1 ? 2.0 / h : (jn == 2 ? -0.5 / h : 0.0));
    if (i == n - 1) return jn == n - 1 ? 1.5 / h : (jn == n - 2 ? -2.0 / h : (jn == n - 3 ? 0.5 / h : 0.0));
    return jn == i + 1 ? 0.5 / h : (jn == i - 1 ? -0.5 / h : 0.0);
}

template <typename AccT, typename OutT>
__global__ void __launch_bounds__(256) k_curl_adjoint(const AccT *__restrict__ acc, int nx, int ny, int nz, double dx,
                                                      double dy, double dz, OutT *__restrict__ dB)
{
    const long long total = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const long long idx[3] = {node % nx, (node / nx) % ny, node / sz};
        const long long n[3] = {nx, ny, nz}, stride[3] = {1, sy, sz};
        const double h[3] = {dx, dy, dz};
        // DT[axis][c] = (D_axis^T dJ_c)(node)
        double DT[3][3];
        for (int a = 0; a < 3; a++) {
            DT[a][0] = DT[a][1] = DT[a][2] = 0.0;
            const long long j0 = idx[a];
            const long long lo = j0 - 2 < 0 ? 0 : j0 - 2, hi = j0 + 2 > n[a] - 1 ? n[a] - 1 : j0 + 2;
            for (long long i = lo; i <= hi; i++) {
                const double cf = stencil(i, j0, n[a], h[a]);
                if (cf == 0.0) continue;
                const AccT *q = acc + 8 * (node + (i - j0) * stride[a]);
                DT[a][0] += cf * (double)q[3];
                DT[a][1] += cf * (double)q[4];
                DT[a][2] += cf * (double)q[5];
            }
        }
        // Jx = Dy Bz - Dz By, Jy = Dz Bx - Dx Bz, Jz = Dx By - Dy Bx
        const AccT *p = acc + 8 * node;
        const double bx = (double)p[0] + DT[2][1] - DT[1][2];
        const double by = (double)p[1] + DT[0][2] - DT[2][0];
        const double bz = (double)p[2] + DT[1][0] - DT[0][1];
        dB[3 * node + 0] = (OutT)((double)dB[3 * node + 0] + bx);
        dB[3 * node + 1] = (OutT)((double)dB[3 * node + 1] + by);
        dB[3 * node + 2] = (OutT)((double)dB[3 * node + 2] + bz);
    }
}

// ---------------------------------------------------------------------------
// loss = mean over usable seeds of (log10 Q - log10 Qt)^2 + w (Tw - Twt)^2
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool usable(long long s, const double *Q, const double *Tw, const double *Qt,
                                       const double *Twt, const uint8_t *st)
{
    const double q = Q[s], qt = Qt[s], t = Tw[s], tt = Twt[s];
    if (st && (st[s] & (kBad | FQSL_LINE_MIXED | FQSL_LINE_ROTATED))) return false;
    return isfinite(q) && isfinite(qt) && isfinite(t) && isfinite(tt) && q > 0.0 && qt > 0.0;
}

__global__ void __launch_bounds__(256) k_loss_sum(long long n, const double *Q, const double *Tw, const double *Qt,
                                                  const double *Twt, const uint8_t *st, double wtw, double *sums)
{
    double s = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (usable(i, Q, Tw, Qt, Twt, st)) {
            const double lq = log10(Q[i]) - log10(Qt[i]);
            const double dt = Tw[i] - Twt[i];
            s += lq * lq + wtw * dt * dt;
            c += 1.0;
        }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    __shared__ double ws[8], wc[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ws[w] = s;
        wc[w] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tc = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            ts += ws[k];
            tc += wc[k];
        }
        atomicAdd(sums, ts);
        atomicAdd(sums + 1, tc);
    }
}

__global__ void __launch_bounds__(256) k_loss_grad(long long n, const double *Q, const double *Tw, const double *Qt,
                                                   const double *Twt, const uint8_t *st, double wtw,
                                                   const double *sums, double *loss, double *dQ, double *dTw)
{
    const double cnt = sums[1] > 0.0 ? sums[1] : 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) *loss = sums[0] / cnt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double gq = 0.0, gt = 0.0;
        if (usable(i, Q, Tw, Qt, Twt, st)) {
            const double lq = log10(Q[i]) - log10(Qt[i]);
            gq = 2.0 * lq / (Q[i] * 2.302585092994046 * cnt);
            gt = 2.0 * wtw * (Tw[i] - Twt[i]) / cnt;
        }
        if (dQ) dQ[i] = gq;
        if (dTw) dTw[i] = gt;
    }
}

// The step sequence of every half-line, in order: ns[hl] steps (-1: more
// than cap; 0 with code -1: line not traced), h[hl * cap + i], end code and the
// chord's exiting step.
template <typename T>
__global__ void __launch_bounds__(256) k_tape_export(const Tape tp, const uint8_t *__restrict__ st, long long halves,
                                                     int cap, int32_t *ns, int32_t *code, double *hx, double *h)
{
    const T *H = (const T *)tp.h;
    for (long long hl = blockIdx.x * (long long)blockDim.x + threadIdx.x; hl < halves;
         hl += (long long)gridDim.x * blockDim.x) {
        ns[hl] = 0;
        code[hl] = -1;
        hx[hl] = 0.0;
        if (st[hl >> 1] & kBad) continue;
        const int4 hd = tp.head[hl];
        if (hd.x < 0 || hd.z < 0) continue;
        long long total = hd.y;
        for (int c = hd.x;;) {
            const int pc = tp.prev[c];
            if (pc < 0 || pc >= c) break;
            total += tp.k;
            c = pc;
        }
        code[hl] = hd.z;
        hx[hl] = (double)((const T *)tp.xe)[4 * hl + 3];
        if (total > cap) {
            ns[hl] = -1;
            continue;
        }
        ns[hl] = (int32_t)total;
        long long pos = total;
        int c = hd.x, m = hd.y;
        for (;;) {
            for (int i = m - 1; i >= 0; i--) h[hl * cap + --pos] = (double)H[(long long)c * tp.k + i];
            const int pc = tp.prev[c];
            if (pc < 0 || pc >= c) break;
            c = pc;
            m = tp.k;
        }
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

unsigned grid_for(long long n, int per_block, int cap_per_sm)
{
    long long b = (n + per_block - 1) / per_block;
    const long long cap = (long long)sm_count() * cap_per_sm;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace adj

// mode: 0 = float state and float grid, 1 = float state and double grid, 2 =
// double; tape_f64: the tape holds doubles (FP64 forward) or floats
namespace {
template <typename TT>
void q_vjp_mode(const AdjArgs &a, int mode, unsigned g, cudaStream_t s)
{
    if (mode == 0) adj::k_q_vjp<float, float, TT><<<g, 128, 0, s>>>(a);
    else if (mode == 1) adj::k_q_vjp<float, double, TT><<<g, 128, 0, s>>>(a);
    else adj::k_q_vjp<double, double, TT><<<g, 128, 0, s>>>(a);
}

template <typename TT>
void reverse_mode(const AdjArgs &a, int mode, int grid, cudaStream_t s)
{
    if (mode == 0) adj::k_reverse<float, float, TT><<<grid, 128, 0, s>>>(a);
    else if (mode == 1) adj::k_reverse<float, double, TT><<<grid, 128, 0, s>>>(a);
    else adj::k_reverse<double, double, TT><<<grid, 128, 0, s>>>(a);
}

template <typename TT>
int reverse_blocks(int mode)
{
    int b = 0;
    if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, adj::k_reverse<float, float, TT>, 128, 0);
    else if (mode == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, adj::k_reverse<float, double, TT>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, adj::k_reverse<double, double, TT>, 128, 0);
    return b > 0 ? b : 1;
}
}  // namespace

cudaError_t launch_q_vjp(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s)
{
    const unsigned g = adj::grid_for(a.n, 128, 16);
    if (tape_f64) q_vjp_mode<double>(a, mode, g, s);
    else q_vjp_mode<float>(a, mode, g, s);
    return cudaGetLastError();
}

int reverse_blocks_per_sm(int mode, bool tape_f64)
{
    return tape_f64 ? reverse_blocks<double>(mode) : reverse_blocks<float>(mode);
}

cudaError_t launch_reverse(const AdjArgs &a, int mode, bool tape_f64, int grid, cudaStream_t s)
{
    if (tape_f64) reverse_mode<double>(a, mode, grid, s);
    else reverse_mode<float>(a, mode, grid, s);
    return cudaGetLastError();
}

cudaError_t launch_curl_adjoint(const void *acc, bool acc64, const FieldView &g, void *dB, fqsl_dtype dt,
                                cudaStream_t s)
{
    const long long total = (long long)g.nx * g.ny * g.nz;
    const unsigned grid = adj::grid_for(total, 256, 8);
    if (acc64) {
        if (dt == FQSL_F32)
            adj::k_curl_adjoint<double, float><<<grid, 256, 0, s>>>((const double *)acc, g.nx, g.ny, g.nz, g.d[0],
                                                                    g.d[1], g.d[2], (float *)dB);
        else
            adj::k_curl_adjoint<double, double><<<grid, 256, 0, s>>>((const double *)acc, g.nx, g.ny, g.nz, g.d[0],
                                                                     g.d[1], g.d[2], (double *)dB);
    } else {
        if (dt == FQSL_F32)
            adj::k_curl_adjoint<float, float><<<grid, 256, 0, s>>>((const float *)acc, g.nx, g.ny, g.nz, g.d[0],
                                                                   g.d[1], g.d[2], (float *)dB);
        else
            adj::k_curl_adjoint<float, double><<<grid, 256, 0, s>>>((const float *)acc, g.nx, g.ny, g.nz, g.d[0],
                                                                    g.d[1], g.d[2], (double *)dB);
    }
    return cudaGetLastError();
}

cudaError_t launch_tape_export(const Tape &tp, bool f64, const uint8_t *st, long long halves, int cap, int32_t *ns,
                               int32_t *code, double *hx, double *h, cudaStream_t s)
{
    const unsigned g = adj::grid_for(halves, 256, 8);
    if (f64) adj::k_tape_export<double><<<g, 256, 0, s>>>(tp, st, halves, cap, ns, code, hx, h);
    else adj::k_tape_export<float><<<g, 256, 0, s>>>(tp, st, halves, cap, ns, code, hx, h);
    return cudaGetLastError();
}

cudaError_t launch_loss(long long n, const double *Q, const double *Tw, const double *Qt, const double *Twt,
                        const uint8_t *st, double wtw, double *sums, double *loss, double *dQ, double *dTw,
                        cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const unsigned g = adj::grid_for(n, 256, 4);
    adj::k_loss_sum<<<g, 256, 0, s>>>(n, Q, Tw, Qt, Twt, st, wtw, sums);
    adj::k_loss_grad<<<g, 256, 0, s>>>(n, Q, Tw, Qt, Twt, st, wtw, sums, loss, dQ, dTw);
    return cudaGetLastError();
}

}  // namespace fqsl
