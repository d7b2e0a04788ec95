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
//                step (Henon step or chord) and every accepted step (RKF45's
//                4th-order solution or the fixed-step scheme's 3/8 rule,
//                stages in reverse), scattering the adjoints of the
//                interpolated B and curl B into a node grid;
//   curl_adjoint per node: dB += dB_interp + curl^T dJ_interp (the transpose
//                of the curl grid's stencils, Eq. tw).
// The state is recomputed in the traced precision T; the node grid
// accumulates in AccT (float with vector atomics, or double).
#include "adjoint.cuh"

namespace fqsl {

namespace adj {


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
template <typename T, typename AccT, bool RECT = false>
__device__ __forceinline__ double bn_vjp(const FieldView &f, const T p[3], int ax, double bnb, double g[3], AccT *acc)
{
    const Cell<T> c = cellg<RECT>(f, p[0], p[1], p[2]);
    g[0] = g[1] = g[2] = 0.0;
    if (!cell_ok(f, c.base)) return 0.0;
    T V[6], dV[3][6];
    interp_d<T, RECT>(f, c, V, dV);
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

// the state coordinates of a physical seed position (a stretched grid's FP64
// state is the physical position itself)
template <typename T, bool RECT>
__device__ __forceinline__ T seed_state(const FieldView &f, double r, int a)
{
    if constexpr (RECT && sizeof(T) == 8) return (T)r;
    else return (T)((r - f.o[a]) / f.d[a]);
}

template <typename T, typename AccT, typename TT, bool RECT = false>
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
        if (st & kBad) continue;
        const double qb = A.dQ ? A.dQ[idx] : 0.0;
        if (!(qb == qb) || qb == 0.0 || fabs(qb) == INFINITY) continue;
        // a rotated seed (Sec. 4) differences its four extra lines over drot
        const bool rot = (st & FQSL_LINE_ROTATED) != 0;
        const int slot = (rot && A.rot_slot) ? A.rot_slot[idx] : 0;
        if (rot && (slot <= 0 || slot > A.n)) continue;
        // lattice index (i, j) within its layer k (each layer is its own S0)
        const long long i = idx % G.n1, j = (idx / G.n1) % G.n2, k = idx / (G.n1 * G.n2);
        long long nid[4];  // neighbour lines (in NR)
        bool has[4];
        if (rot) {
            for (int q = 0; q < 4; q++) {
                nid[q] = 4LL * (slot - 1) + q;
                has[q] = true;
            }
        } else {
            const long long ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
            for (int q = 0; q < 4; q++) {
                has[q] = ni[q] >= 0 && ni[q] < G.n1 && nj[q] >= 0 && nj[q] < G.n2;
                nid[q] = has[q] ? ni[q] + G.n1 * (nj[q] + G.n2 * k) : 0;
            }
        }
        const LineRecs &NR = rot ? A.ext : R;
        const long long hbase = rot ? 2 * A.n : 0;  // half-line of NR's line 0
        const double inv[2] = {rot ? 1.0 / G.drot : 1.0 / G.du, rot ? 1.0 / G.drot : 1.0 / G.dv};
        const int fe2[2] = {R.f1[idx], R.f2[idx]};
        // J_e[r][s] = sum over two half-lines of cf * xi_{ra[r]}(half-line)
        double Jm[2][2][2];
        long long ln[2][2][2];  // [e][s][plus/minus]: half-line
        double cf[2][2][2];     // the two coefficients (index units; times d below)
        bool mixed = false;
        for (int e = 0; e < 2 && !mixed; e++) {
            int ra[2];
            face_axes(fe2[e], ra[0], ra[1]);
            for (int s = 0; s < 2 && !mixed; s++) {
                const int P = 2 * s, M = 2 * s + 1;
                const bool okp = has[P] && !(NR.st[nid[P]] & kBad) && (e == 0 ? NR.f1 : NR.f2)[nid[P]] == fe2[e];
                const bool okm = has[M] && !(NR.st[nid[M]] & kBad) && (e == 0 ? NR.f1 : NR.f2)[nid[M]] == fe2[e];
                const long long hp = hbase + 2 * nid[P] + e, hm = hbase + 2 * nid[M] + e, h0 = 2 * idx + e;
                if (okp && okm) {
                    ln[e][s][0] = hp;
                    ln[e][s][1] = hm;
                    cf[e][s][0] = 0.5 * inv[s];
                    cf[e][s][1] = -0.5 * inv[s];
                } else if (okp) {
                    ln[e][s][0] = hp;
                    ln[e][s][1] = h0;
                    cf[e][s][0] = inv[s];
                    cf[e][s][1] = -inv[s];
                } else if (okm) {
                    ln[e][s][0] = h0;
                    ln[e][s][1] = hm;
                    cf[e][s][0] = inv[s];
                    cf[e][s][1] = -inv[s];
                } else {
                    mixed = true;
                    break;
                }
                for (int r = 0; r < 2; r++) {
                    const int a = ra[r];
                    const double xp = (double)XE[4 * ln[e][s][0] + a];
                    const double xm = (double)XE[4 * ln[e][s][1] + a];
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
        const double bn1 = bn_vjp<T, AccT, RECT>(f, pe[0], ax1, 0.0, g1, acc);
        const double bn2 = bn_vjp<T, AccT, RECT>(f, pe[1], ax2, 0.0, g2, acc);
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
                    atomicAdd(A.xbar + 3 * ln[e][s][0] + a, cf[e][s][0] * v);
                    atomicAdd(A.xbar + 3 * ln[e][s][1] + a, cf[e][s][1] * v);
                }
        }
        // |Bn1 Bn2| / Bn0^2
        const double sg1 = bn1 < 0.0 ? -1.0 : 1.0, sg2 = bn2 < 0.0 ? -1.0 : 1.0;
        const double bn1b = sb * sg1 * fabs(bn2) / (bn0 * bn0);
        const double bn2b = sb * sg2 * fabs(bn1) / (bn0 * bn0);
        const double bn0b = -2.0 * sb * fabs(bn1 * bn2) / (bn0 * bn0 * bn0);
        bn_vjp<T, AccT, RECT>(f, pe[0], ax1, bn1b, g1, acc);
        bn_vjp<T, AccT, RECT>(f, pe[1], ax2, bn2b, g2, acc);
        for (int a = 0; a < 3; a++) {
            atomicAdd(A.xbar + 3 * (2 * idx + 0) + a, bn1b * g1[a]);
            atomicAdd(A.xbar + 3 * (2 * idx + 1) + a, bn2b * g2[a]);
        }
        // Bn0 = B(seed) . n0, or |B(seed)| for a rotated seed
        T p0[3];
        if (A.prep.seed) {
            // the FP32 tracer's seed (its pre-pass)
            const float4 sd = A.prep.seed[idx];
            p0[0] = (T)sd.x;
            p0[1] = (T)sd.y;
            p0[2] = (T)sd.z;
        } else {
            // the FP64 tracer's seed: (r0 - o)/d as written (on a stretched
            // grid the physical seed)
            double r0[3];
            trace::lattice_seed(G, i, j, k, r0);
            for (int a = 0; a < 3; a++) p0[a] = seed_state<T, RECT>(f, r0[a], a);
        }
        const Cell<T> c0 = cellg<RECT>(f, p0[0], p0[1], p0[2]);
        if (!cell_ok(f, c0.base)) continue;
        double nb[3] = {G.n0[0], G.n0[1], G.n0[2]};
        if (rot) {
            T V[6], dV[3][6];
            interp_d<T, RECT>(f, c0, V, dV);
            const double B0[3] = {(double)V[0], (double)V[1], (double)V[2]};
            const double nB = sqrt(B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2]);
            if (!(nB > 0.0)) continue;
            for (int a = 0; a < 3; a++) nb[a] = B0[a] / nB;
        }
        const T Vb[6] = {(T)(bn0b * nb[0]), (T)(bn0b * nb[1]), (T)(bn0b * nb[2]), 0, 0, 0};
        scatter(f, c0, Vb, acc);
    }
}

// The extra lines of a rotated seed start at r0 +- drot u and r0 +- drot v,
// where (u, v) = perp_frame(B(r0)/|B(r0)|) (Sec. 4): the adjoints of their
// seeds (pass B) are carried back through the frame to B at the seed's cell.
// u = t/|t| with t = bhat x e_m (m: the smallest |bhat_m|, held fixed), v =
// bhat x u. One thread per rotated seed.
template <typename T, typename AccT, bool RECT = false>
__global__ void __launch_bounds__(128) k_frame_vjp(const AdjArgs A)
{
    const Lattice &G = A.lat;
    const FieldView &f = A.f;
    AccT *acc = (AccT *)A.acc;
    long long nrot = (long long)*A.rot_count;
    if (nrot > A.n) nrot = A.n;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nrot;
         s += (long long)gridDim.x * blockDim.x) {
        // adjoints of the four extra seeds (physical coordinates): both
        // half-lines of a line start at its seed
        double rb[4][3];
        bool any = false;
        for (int q = 0; q < 4; q++) {
            const double *x0 = A.xseed + 3 * (2 * (4 * s + q));
            for (int a = 0; a < 3; a++) {
                rb[q][a] = (x0[a] + x0[3 + a]) / f.d[a];
                any = any || rb[q][a] != 0.0;
            }
        }
        if (!any) continue;
        const long long idx = A.rot_seed[s];
        if (idx < 0 || idx >= A.n) {
            record_fail(f.err, 4, idx);
            continue;
        }
        const long long i = idx % G.n1, j = (idx / G.n1) % G.n2, k = idx / (G.n1 * G.n2);
        double r0[3];
        T xi[3];
        trace::lattice_seed(G, i, j, k, r0);
        for (int a = 0; a < 3; a++) xi[a] = seed_state<T, RECT>(f, r0[a], a);
        const Cell<T> c = cellg<RECT>(f, xi[0], xi[1], xi[2]);
        if (!cell_ok(f, c.base)) continue;
        T V[6], dV[3][6];
        interp_d<T, RECT>(f, c, V, dV);
        const double B0[3] = {(double)V[0], (double)V[1], (double)V[2]};
        const double nB = sqrt(B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2]);
        if (!(nB > 0.0)) continue;
        const double bh[3] = {B0[0] / nB, B0[1] / nB, B0[2] / nB};
        int m = 0;
        if (fabs(bh[1]) < fabs(bh[m])) m = 1;
        if (fabs(bh[2]) < fabs(bh[m])) m = 2;
        const int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
        // t = bhat x e_m: t_m = 0, t_m1 = bhat_m2, t_m2 = -bhat_m1
        double t[3];
        t[m] = 0.0;
        t[m1] = bh[m2];
        t[m2] = -bh[m1];
        const double nt = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        const double u[3] = {t[0] / nt, t[1] / nt, t[2] / nt};
        // seeds r0 + sg drot dir: ubar, vbar
        double ub[3], vb[3];
        for (int a = 0; a < 3; a++) {
            ub[a] = G.drot * (rb[0][a] - rb[1][a]);
            vb[a] = G.drot * (rb[2][a] - rb[3][a]);
        }
        // v = bhat x u: bhat_bar = u x vbar, ubar += vbar x bhat
        double bhb[3] = {u[1] * vb[2] - u[2] * vb[1], u[2] * vb[0] - u[0] * vb[2], u[0] * vb[1] - u[1] * vb[0]};
        ub[0] += vb[1] * bh[2] - vb[2] * bh[1];
        ub[1] += vb[2] * bh[0] - vb[0] * bh[2];
        ub[2] += vb[0] * bh[1] - vb[1] * bh[0];
        // u = t/|t|: tbar = (ubar - u (u . ubar))/|t|
        const double uu = u[0] * ub[0] + u[1] * ub[1] + u[2] * ub[2];
        double tb[3];
        for (int a = 0; a < 3; a++) tb[a] = (ub[a] - u[a] * uu) / nt;
        // t = bhat x e_m: bhat_bar += e_m x tbar
        bhb[m1] += -tb[m2];
        bhb[m2] += tb[m1];
        // bhat = B0/|B0|
        const double bb = bh[0] * bhb[0] + bh[1] * bhb[1] + bh[2] * bhb[2];
        const T Vb[6] = {(T)((bhb[0] - bh[0] * bb) / nB), (T)((bhb[1] - bh[1] * bb) / nB),
                         (T)((bhb[2] - bh[2] * bb) / nB), 0, 0, 0};
        scatter(f, c, Vb, acc);
    }
}

// ---------------------------------------------------------------------------
// dB += dB_interp + curl^T dJ_interp (per node)
// ---------------------------------------------------------------------------
// coefficient of node jn in row i of the curl grid's derivative stencil along
// an axis of n nodes, rh = 1/spacing
template <typename A>
__device__ __forceinline__ A stencil(int i, int jn, int n, A rh)
{
    if (n == 2) return jn == 1 ? rh : -rh;
    if (i == 0) return jn == 0 ? (A)-1.5 * rh : (jn == 1 ? (A)2 * rh : (jn == 2 ? (A)-0.5 * rh : (A)0));
    if (i == n - 1) return jn == n - 1 ? (A)1.5 * rh : (jn == n - 2 ? (A)-2 * rh : (jn == n - 3 ? (A)0.5 * rh : (A)0));
    return jn == i + 1 ? (A)0.5 * rh : (jn == i - 1 ? (A)-0.5 * rh : (A)0);
}

template <typename AccT, typename OutT>
__global__ void __launch_bounds__(256) k_curl_adjoint(const AccT *__restrict__ acc, int nx, int ny, int nz, double dx,
                                                      double dy, double dz, OutT *__restrict__ dB)
{
    const long long total = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    // half reciprocal spacings for the central rows, in the grid's precision
    const AccT hx = (AccT)(0.5 / dx), hy = (AccT)(0.5 / dy), hz = (AccT)(0.5 / dz);
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const unsigned un = (unsigned)node, uxy = (unsigned)nx * (unsigned)ny;  // nodes < 2^31
        const unsigned iz = un / uxy, rem = un - iz * uxy, iy = rem / (unsigned)nx, ix = rem - iy * (unsigned)nx;
        const long long n[3] = {nx, ny, nz}, stride[3] = {1, sy, sz};
        const int idx[3] = {(int)ix, (int)iy, (int)iz};
        const AccT hh[3] = {hx, hy, hz};
        // DT[axis][c] = (D_axis^T dJ_c)(node)
        AccT DT[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int j0 = idx[a];
            if (j0 >= 3 && j0 + 3 < n[a]) {
                // only the central rows j0 -+ 1 reach this node: coefficients -+1/(2h)
                const AccT *qm = acc + 8 * (node - stride[a]);
                const AccT *qp = acc + 8 * (node + stride[a]);
                DT[a][0] = hh[a] * (qm[3] - qp[3]);
                DT[a][1] = hh[a] * (qm[4] - qp[4]);
                DT[a][2] = hh[a] * (qm[5] - qp[5]);
            } else {
                // rows near the faces (the one-sided stencils of the curl grid)
                AccT t0 = 0, t1 = 0, t2 = 0;
                const int na = (int)n[a];
                const int lo = j0 - 2 < 0 ? 0 : j0 - 2, hi = j0 + 2 > na - 1 ? na - 1 : j0 + 2;
                for (int i = lo; i <= hi; i++) {
                    const AccT cf = stencil<AccT>(i, j0, na, (AccT)2 * hh[a]);
                    if (cf == (AccT)0) continue;
                    const AccT *q = acc + 8 * (node + (long long)(i - j0) * stride[a]);
                    t0 += cf * q[3];
                    t1 += cf * q[4];
                    t2 += cf * q[5];
                }
                DT[a][0] = t0;
                DT[a][1] = t1;
                DT[a][2] = t2;
            }
        }
        // Jx = Dy Bz - Dz By, Jy = Dz Bx - Dx Bz, Jz = Dx By - Dy Bx
        const AccT *p = acc + 8 * node;
        const AccT bx = p[0] + DT[2][1] - DT[1][2];
        const AccT by = p[1] + DT[0][2] - DT[2][0];
        const AccT bz = p[2] + DT[1][0] - DT[0][1];
        using W = decltype(AccT{} + OutT{});  // the wider of the two
        dB[3 * node + 0] = (OutT)((W)dB[3 * node + 0] + (W)bx);
        dB[3 * node + 1] = (OutT)((W)dB[3 * node + 1] + (W)by);
        dB[3 * node + 2] = (OutT)((W)dB[3 * node + 2] + (W)bz);
    }
}

// The same on a stretched grid: the curl grid's derivative along an axis of n
// nodes at row i is the three-point stencil of a non-uniform axis with the
// coefficients co[3 i ..] (field.cu): interior rows on nodes i-1, i, i+1; row 0
// on nodes 0, 1, 2 (third coefficient negated); row n-1 on nodes n-3, n-2, n-1
// (second negated); (f1 - f0)/(x1 - x0) on an axis of 2 nodes. Coefficient of
// node jn in row i:
__device__ __forceinline__ double stencil_rect(int i, int jn, int n, const double *__restrict__ X,
                                               const double *__restrict__ co)
{
    if (n == 2) return (jn == 1 ? 1.0 : -1.0) / (X[1] - X[0]);
    const double c0 = co[3 * i], c1 = co[3 * i + 1], c2 = co[3 * i + 2];
    if (i == 0) return jn == 0 ? c0 : (jn == 1 ? c1 : (jn == 2 ? -c2 : 0.0));
    if (i == n - 1) return jn == n - 3 ? c0 : (jn == n - 2 ? -c1 : (jn == n - 1 ? c2 : 0.0));
    return jn == i - 1 ? c0 : (jn == i ? c1 : (jn == i + 1 ? c2 : 0.0));
}

template <typename AccT, typename OutT>
__global__ void __launch_bounds__(256) k_curl_adjoint_rect(const AccT *__restrict__ acc, const FieldView g,
                                                           OutT *__restrict__ dB)
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long total = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(node % nx), iy = (int)((node / nx) % ny), iz = (int)(node / sz);
        const int n[3] = {nx, ny, nz}, idx[3] = {ix, iy, iz};
        const long long stride[3] = {1, sy, sz};
        // DT[axis][c] = (D_axis^T dJ_c)(node): the rows whose stencil reaches this node
        AccT DT[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            AccT t0 = 0, t1 = 0, t2 = 0;
            const int j0 = idx[a], na = n[a];
            const int lo = j0 - 2 < 0 ? 0 : j0 - 2, hi = j0 + 2 > na - 1 ? na - 1 : j0 + 2;
            for (int i = lo; i <= hi; i++) {
                const AccT cf = (AccT)stencil_rect(i, j0, na, g.x64[a], g.dco[a]);
                if (cf == (AccT)0) continue;
                const AccT *q = acc + 8 * (node + (long long)(i - j0) * stride[a]);
                t0 += cf * q[3];
                t1 += cf * q[4];
                t2 += cf * q[5];
            }
            DT[a][0] = t0;
            DT[a][1] = t1;
            DT[a][2] = t2;
        }
        // Jx = Dy Bz - Dz By, Jy = Dz Bx - Dx Bz, Jz = Dx By - Dy Bx
        const AccT *p = acc + 8 * node;
        const AccT bx = p[0] + DT[2][1] - DT[1][2];
        const AccT by = p[1] + DT[0][2] - DT[2][0];
        const AccT bz = p[2] + DT[1][0] - DT[0][1];
        using W = decltype(AccT{} + OutT{});
        dB[3 * node + 0] = (OutT)((W)dB[3 * node + 0] + (W)bx);
        dB[3 * node + 1] = (OutT)((W)dB[3 * node + 1] + (W)by);
        dB[3 * node + 2] = (OutT)((W)dB[3 * node + 2] + (W)bz);
    }
}

// ---------------------------------------------------------------------------
// loss = mean over usable seeds of (log10 Q - log10 Qt)^2 + w (Tw - Twt)^2
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool usable(long long s, const double *Q, const double *Tw, const double *Qt,
                                       const double *Twt, const uint8_t *st)
{
    const double q = Q[s], qt = Qt[s], t = Tw[s], tt = Twt[s];
    if (st && (st[s] & (kBad | FQSL_LINE_MIXED))) return false;
    return isfinite(q) && isfinite(qt) && isfinite(t) && isfinite(tt) && q > 0.0 && qt > 0.0;
}

// The misfit sums; with lq_out/dt_out (the gradient's buffers) each usable
// seed's log-Q difference and Tw difference are kept there for k_loss_grad,
// so that the FP64 logarithms (the costly part on GB300's FP64 pipe) are
// taken once.
__global__ void __launch_bounds__(256) k_loss_sum(long long n, const double *Q, const double *Tw, const double *Qt,
                                                  const double *Twt, const uint8_t *st, double wtw, double *sums,
                                                  double *lq_out, double *dt_out)
{
    double s = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (usable(i, Q, Tw, Qt, Twt, st)) {
            const double lq = log10(Q[i]) - log10(Qt[i]);
            const double dt = Tw[i] - Twt[i];
            if (lq_out) {
                lq_out[i] = lq;
                dt_out[i] = dt;
            }
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
                                                   const double *sums, double *loss, double *dQ, double *dTw,
                                                   bool keep)
{
    const double cnt = sums[1] > 0.0 ? sums[1] : 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) *loss = sums[0] / cnt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double gq = 0.0, gt = 0.0;
        if (usable(i, Q, Tw, Qt, Twt, st)) {
            // dQ, dTw hold k_loss_sum's differences when it kept them
            const double lq = keep ? dQ[i] : log10(Q[i]) - log10(Qt[i]);
            const double dt = keep ? dTw[i] : Tw[i] - Twt[i];
            gq = 2.0 * lq / (Q[i] * 2.302585092994046 * cnt);
            gt = 2.0 * wtw * dt / cnt;
        }
        if (dQ) dQ[i] = gq;
        if (dTw) dTw[i] = gt;
    }
}

// The step sequence of every half-line, in order: ns[hl] steps (0 with code
// -1: line not traced), h[hl * cap + i] when ns[hl] <= cap, end code and the
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
        ns[hl] = (int32_t)total;
        if (total > cap) continue;
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

// stretched grids: the forward's state convention (FP64 physical, FP32
// relative to the first node) is the reverse sweep's, so the tape and the
// sweep share their precision (the host enforces it)
void q_vjp_rect(const AdjArgs &a, int mode, unsigned g, cudaStream_t s)
{
    if (mode == 0) adj::k_q_vjp<float, float, float, true><<<g, 128, 0, s>>>(a);
    else if (mode == 1) adj::k_q_vjp<float, double, float, true><<<g, 128, 0, s>>>(a);
    else adj::k_q_vjp<double, double, double, true><<<g, 128, 0, s>>>(a);
}

template <typename T, typename AccT, bool RECT = false>
void frame_pass(const AdjArgs &a, cudaStream_t s)
{
    if (a.rot_count) adj::k_frame_vjp<T, AccT, RECT><<<adj::grid_for(a.n, 128, 4), 128, 0, s>>>(a);
}

template <typename TT>
void reverse_mode(const AdjArgs &a, int mode, cudaStream_t s)
{
    if (mode == 0) adj::reverse_passes<float, float, TT, 0>(a, s);
    else if (mode == 1) adj::reverse_passes<float, double, TT, 0>(a, s);
    else adj::reverse_passes<double, double, TT, 0>(a, s);
}
}  // namespace

cudaError_t launch_q_vjp(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s)
{
    const unsigned g = adj::grid_for(a.n, 128, 16);
    if (a.f.rect) q_vjp_rect(a, mode, g, s);
    else if (tape_f64) q_vjp_mode<double>(a, mode, g, s);
    else q_vjp_mode<float>(a, mode, g, s);
    return cudaGetLastError();
}

cudaError_t launch_reverse(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s)
{
    if (a.chunks > 0 && a.f.rect) {
        const cudaError_t e = launch_reverse_rect(a, mode, s);
        if (e != cudaSuccess) return e;
        if (mode == 0) frame_pass<float, float, true>(a, s);
        else if (mode == 1) frame_pass<float, double, true>(a, s);
        else frame_pass<double, double, true>(a, s);
    } else if (a.chunks > 0) {
        if (a.p.scheme == 1) {
            const cudaError_t e = launch_reverse_rk38(a, mode, tape_f64, s);
            if (e != cudaSuccess) return e;
        } else if (tape_f64) {
            reverse_mode<double>(a, mode, s);
        } else {
            reverse_mode<float>(a, mode, s);
        }
        // the frames of rotated seeds, after every half-line's seed adjoint
        if (mode == 0) frame_pass<float, float>(a, s);
        else if (mode == 1) frame_pass<float, double>(a, s);
        else frame_pass<double, double>(a, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_curl_adjoint(const void *acc, bool acc64, const FieldView &g, void *dB, fqsl_dtype dt,
                                cudaStream_t s)
{
    const long long total = (long long)g.nx * g.ny * g.nz;
    const unsigned grid = adj::grid_for(total, 256, 8);
    if (g.rect) {
        if (acc64) {
            if (dt == FQSL_F32)
                adj::k_curl_adjoint_rect<double, float><<<grid, 256, 0, s>>>((const double *)acc, g, (float *)dB);
            else
                adj::k_curl_adjoint_rect<double, double><<<grid, 256, 0, s>>>((const double *)acc, g, (double *)dB);
        } else {
            if (dt == FQSL_F32)
                adj::k_curl_adjoint_rect<float, float><<<grid, 256, 0, s>>>((const float *)acc, g, (float *)dB);
            else
                adj::k_curl_adjoint_rect<float, double><<<grid, 256, 0, s>>>((const float *)acc, g, (double *)dB);
        }
        return cudaGetLastError();
    }
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
    // (not when an output buffer is also an input: the kept differences would
    // overwrite it before k_loss_grad reads it)
    const double *ins[4] = {Q, Tw, Qt, Twt};
    bool keep = dQ && dTw && dQ != dTw;
    for (const double *in : ins) keep = keep && in != dQ && in != dTw;
    adj::k_loss_sum<<<g, 256, 0, s>>>(n, Q, Tw, Qt, Twt, st, wtw, sums, keep ? dQ : nullptr, keep ? dTw : nullptr);
    adj::k_loss_grad<<<g, 256, 0, s>>>(n, Q, Tw, Qt, Twt, st, wtw, sums, loss, dQ, dTw, keep);
    return cudaGetLastError();
}

}  // namespace fqsl
