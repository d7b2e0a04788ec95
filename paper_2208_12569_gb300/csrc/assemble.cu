// q_assemble: Method I squashing factor from neighbouring footpoints.
//
// For each lattice seed the footpoint maps of both ends are differenced over
// the lattice neighbours (or the four extra lines of a rotated S0): J_e =
// d(face coordinates of end e)/d(S0 coordinates), central differences when
// both neighbours end on the centre's face, one-sided when one does, NaN and
// FQSL_LINE_MIXED otherwise (Sec. 2.1: Code2016 gave NaN). Then Eq. D+-2 with
// Eq. D+-3 and Eq. Q+- with |det D| replaced by |Bn1/Bn2| (Eq. Bn1) give
//   Q = |J2 adj(J1)|_F^2 |Bn1 Bn2| / Bn0^2.
// All of it in FP64. One thread per seed; the neighbours' records are shared
// through L1/L2, so the kernel streams the line records once (HBM-bound).
#include <math.h>

#include "fqsl_internal.cuh"

namespace fqsl {
namespace {

__device__ __forceinline__ void face_coords(const double *r, int face, double fc[2])
{
    const int a = face >> 1;
    fc[0] = (a == 0) ? r[1] : r[0];
    fc[1] = (a == 2) ? r[1] : r[2];
}

}  // namespace

__device__ __forceinline__ void assemble_one_f64(const AssembleArgs &A, long long idx)
{
    const Lattice &G = A.lat;
    {
        const LineRecs &R = A.rec;
        unsigned st = R.st[idx];
        double Q = NAN;
        if (A.want_q && !(st & kBad)) {
            const long long i = idx % G.n1, j = (idx / G.n1) % G.n2, k = idx / (G.n1 * G.n2);
            const int slot = A.rot_slot ? A.rot_slot[idx] : 0;
            const LineRecs *NR = slot > 0 ? &A.ext : &A.rec;
            long long nid[4];
            bool has[4];
            double du = G.du, dv = G.dv;
            if (slot > 0) {
                for (int q = 0; q < 4; q++) {
                    nid[q] = (long long)(slot - 1) * 4 + q;
                    has[q] = true;
                }
                du = dv = G.drot;
            } else {
                const long long ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
                for (int q = 0; q < 4; q++) {
                    has[q] = ni[q] >= 0 && ni[q] < G.n1 && nj[q] >= 0 && nj[q] < G.n2;
                    nid[q] = ni[q] + G.n1 * (nj[q] + G.n2 * k);
                }
            }
            double Jm[2][2][2];
            bool mixed = false;
            for (int e = 0; e < 2 && !mixed; e++) {
                const int fe = (e == 0 ? R.f1 : R.f2)[idx];
                double f0[2], fp[2], fm[2];
                face_coords((e == 0 ? R.r1 : R.r2) + 3 * idx, fe, f0);
                for (int s = 0; s < 2 && !mixed; s++) {
                    const int P = 2 * s, M = 2 * s + 1;
                    const double del = s ? dv : du;
                    bool okp = false, okm = false;
                    if (has[P]) {
                        const long long id = nid[P];
                        okp = !(NR->st[id] & kBad) && (e == 0 ? NR->f1 : NR->f2)[id] == fe;
                        if (okp) face_coords((e == 0 ? NR->r1 : NR->r2) + 3 * id, fe, fp);
                    }
                    if (has[M]) {
                        const long long id = nid[M];
                        okm = !(NR->st[id] & kBad) && (e == 0 ? NR->f1 : NR->f2)[id] == fe;
                        if (okm) face_coords((e == 0 ? NR->r1 : NR->r2) + 3 * id, fe, fm);
                    }
                    for (int r = 0; r < 2; r++) {
                        if (okp && okm) Jm[e][r][s] = (fp[r] - fm[r]) / (2.0 * del);
                        else if (okp) Jm[e][r][s] = (fp[r] - f0[r]) / del;
                        else if (okm) Jm[e][r][s] = (f0[r] - fm[r]) / del;
                        else mixed = true;
                    }
                }
            }
            if (mixed) {
                st |= FQSL_LINE_MIXED;
            } else {
                // D12 = J2 adj(J1) / |Bn0/Bn1|  (Eqs. D+-2, D+-3)
                const double adj[2][2] = {{Jm[0][1][1], -Jm[0][0][1]}, {-Jm[0][1][0], Jm[0][0][0]}};
                double norm2 = 0.0;
                for (int r = 0; r < 2; r++)
                    for (int s = 0; s < 2; s++) {
                        const double m = Jm[1][r][0] * adj[0][s] + Jm[1][r][1] * adj[1][s];
                        norm2 += m * m;
                    }
                const double bn0 = R.bn0[idx];
                Q = norm2 * fabs(R.bn1[idx] * R.bn2[idx]) / (bn0 * bn0);
            }
        }
        const fqsl_out &o = A.out;
        const bool bad = (st & kBad) != 0;
        if (o.Q) o.Q[idx] = Q;
        if (o.Tw) o.Tw[idx] = bad ? NAN : R.tw[idx];
        if (o.length) o.length[idx] = bad ? NAN : R.len[idx];
        if (o.r1)
            for (int c = 0; c < 3; c++) o.r1[3 * idx + c] = R.r1[3 * idx + c];
        if (o.r2)
            for (int c = 0; c < 3; c++) o.r2[3 * idx + c] = R.r2[3 * idx + c];
        if (o.face1) o.face1[idx] = R.f1[idx];
        if (o.face2) o.face2[idx] = R.f2[idx];
        if (o.status) o.status[idx] = (uint8_t)st;
        if (o.steps) o.steps[idx] = R.steps[idx];
    }
}

namespace {

__global__ void __launch_bounds__(256) k_assemble(const AssembleArgs A)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
         idx += (long long)gridDim.x * blockDim.x)
        assemble_one_f64(A, idx);
}

__device__ __forceinline__ double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Method II (Sec. 2.1, Eq. q_scott with absolute values): at each end the
// deviation vectors are projected onto the exit face along B, U~ = U -
// (U.n)/(B.n) B, and Q = |U~1^2 V~2^2 + U~2^2 V~1^2 - 2 (U~1.V~1)(U~2.V~2)|
// |Bn1 Bn2| / Bn0^2 with Bn0 = |B| at the seed (S0 perpendicular to B).
// Q_perp (qperp): the end planes perpendicular to B, n = B/|B| at each end.
__global__ void __launch_bounds__(256) k_assemble_m2(const AssembleArgs A)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
         idx += (long long)gridDim.x * blockDim.x) {
        const LineRecs &R = A.rec;
        const unsigned st = R.st[idx];
        const bool bad = (st & kBad) != 0;
        double Q = NAN;
        if (!bad) {
            double Ut[2][3], Vt[2][3], bn[2];
            for (int e = 0; e < 2; e++) {
                const int a = (e == 0 ? R.f1 : R.f2)[idx] >> 1;
                const double *U = R.dev64 + 12 * idx + 6 * e, *V = U + 3, *B = R.be64 + 6 * idx + 3 * e;
                if (A.qperp) {
                    // Q_perp: the end plane perpendicular to B, n = B/|B|
                    const double BB = dot3(B, B), ub = dot3(U, B) / BB, vb = dot3(V, B) / BB;
                    bn[e] = sqrt(BB);
                    for (int b = 0; b < 3; b++) {
                        Ut[e][b] = U[b] - ub * B[b];
                        Vt[e][b] = V[b] - vb * B[b];
                    }
                    continue;
                }
                bn[e] = B[a];
                for (int b = 0; b < 3; b++) {
                    Ut[e][b] = U[b] - U[a] / B[a] * B[b];
                    Vt[e][b] = V[b] - V[a] / B[a] * B[b];
                }
            }
            const double num = dot3(Ut[0], Ut[0]) * dot3(Vt[1], Vt[1]) + dot3(Ut[1], Ut[1]) * dot3(Vt[0], Vt[0]) -
                               2.0 * dot3(Ut[0], Vt[0]) * dot3(Ut[1], Vt[1]);
            const double bn0 = R.bn0[idx];
            Q = fabs(num) * fabs(bn[0] * bn[1]) / (bn0 * bn0);
        }
        const fqsl_out &o = A.out;
        if (o.Q) o.Q[idx] = Q;
        if (o.Tw) o.Tw[idx] = bad ? NAN : R.tw[idx];
        if (o.length) o.length[idx] = bad ? NAN : R.len[idx];
        if (o.r1)
            for (int c = 0; c < 3; c++) o.r1[3 * idx + c] = R.r1[3 * idx + c];
        if (o.r2)
            for (int c = 0; c < 3; c++) o.r2[3 * idx + c] = R.r2[3 * idx + c];
        if (o.face1) o.face1[idx] = R.f1[idx];
        if (o.face2) o.face2[idx] = R.f2[idx];
        if (o.status) o.status[idx] = (uint8_t)st;
        if (o.steps) o.steps[idx] = R.steps[idx];
    }
}

}  // namespace

cudaError_t launch_assemble_m2_f64(const AssembleArgs &a, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (a.n + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    k_assemble_m2<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

namespace {
// entry b of a batch holding item idx: nbase[b] <= idx < nbase[b + 1]
__device__ __forceinline__ int batch_entry(const long long *__restrict__ base, int nent, long long idx)
{
    int lo = 0, hi = nent - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_batch_assemble_f64(const AssembleArgs *__restrict__ desc,
                                                            const long long *__restrict__ nbase, int nent)
{
    const long long total = nbase[nent];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = batch_entry(nbase, nent, idx);
        assemble_one_f64(desc[b], idx - nbase[b]);
    }
}
}  // namespace

cudaError_t launch_batch_assemble_f64(const AssembleArgs *desc, const long long *nbase, int nent, long long total,
                                      cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    k_batch_assemble_f64<<<(unsigned)blocks, 256, 0, s>>>(desc, nbase, nent);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const AssembleArgs &a, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (a.n + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_assemble<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fqsl
