// q_assemble for the FP32 tracers: the FP32 tracer leaves index-space
// footpoints, exit faces and compensated length/Tw partial sums; this kernel
// forms, with every thread of a warp busy, the physical footpoints, the length
// and Tw totals (Eq. tw) and Method I's Q (Eqs. D+-2, D+-3, Q+- with
// |det D| -> |Bn1/Bn2|, Eq. Bn1) in FP64: J_e = d(face coordinates)/d(S0
// coordinates) by central differences when both neighbours end on the
// centre's face, one-sided when one does, NaN and FQSL_LINE_MIXED otherwise.
// Neighbouring footpoints are differenced in index space first (exact for
// nearby values in float) and scaled by the spacing in FP64. Bn at both ends
// is trilinear in the FP32 records (Sec. 2.2), and the factor |Bn1 Bn2|/Bn0^2
// is formed as two correctly rounded float quotients (its inputs are floats;
// GB300's FP64 pipe is the kernel's bound). On a stretched
// grid the FP32 state is the physical position relative to the first node
// (the field view's origin, with unit spacing), so the same forms apply.
#include <math.h>

#include "bits.cuh"
#include "trace.cuh"

namespace fqsl {
namespace {

// the two non-normal axes of a face, in increasing order
__device__ __forceinline__ void face_axes(int face, int &r0, int &r1)
{
    const int a = face >> 1;
    r0 = (a == 0) ? 1 : 0;
    r1 = (a == 2) ? 1 : 2;
}

// Bn of a footpoint on its exit face, trilinear in the FP32 records
__device__ __forceinline__ float bn_at(const FieldView &f, const float *xi, int face)
{
    float B[3], J[3];
    if (f.rect) trace::gather_rect(f, xi[0], xi[1], xi[2], B, J);
    else trace::gather(f, xi[0], xi[1], xi[2], B, J);
    const int a = face >> 1;
    return a == 0 ? B[0] : (a == 1 ? B[1] : B[2]);
}

}  // namespace

__device__ __forceinline__ void assemble_one_f32(const AssembleArgs &A, long long idx)
{
    const Lattice &G = A.lat;
    const FieldView &f = A.f;
    {
        const LineRecs &R = A.rec;
        unsigned st = R.st[idx];
        const bool bad = (st & kBad) != 0;
        const float *x1 = R.xi1 + 3 * idx, *x2 = R.xi2 + 3 * idx;
        const int f1 = R.f1[idx], f2 = R.f2[idx];
        double Q = NAN;
        if (A.want_q && !bad) {
            // 32-bit index arithmetic (a lattice holds fewer than 2^31 seeds)
            const unsigned u = (unsigned)idx, n1 = (unsigned)G.n1, n12 = (unsigned)(G.n1 * G.n2);
            const unsigned k = u / n12, rem = u - k * n12, j = rem / n1, i = rem - j * n1;
            const int slot = A.rot_slot ? A.rot_slot[idx] : 0;
            const LineRecs *NR = slot > 0 ? &A.ext : &A.rec;
            long long nid[4];
            bool has[4];
            // spacing over lattice step per axis (host-computed: no FP64 division here)
            const double *sc[2] = {G.sdu, G.sdv};
            if (slot > 0) {
                for (int q = 0; q < 4; q++) {
                    nid[q] = (long long)(slot - 1) * 4 + q;
                    has[q] = true;
                }
                sc[0] = sc[1] = G.sdr;
            } else {
                const long long ii = i, jj = j, kk = k;
                const long long ni[4] = {ii + 1, ii - 1, ii, ii}, nj[4] = {jj, jj, jj + 1, jj - 1};
                for (int q = 0; q < 4; q++) {
                    has[q] = ni[q] >= 0 && ni[q] < G.n1 && nj[q] >= 0 && nj[q] < G.n2;
                    nid[q] = ni[q] + G.n1 * (nj[q] + G.n2 * kk);
                }
            }
            double Jm[2][2][2];
            bool mixed = false;
            for (int e = 0; e < 2 && !mixed; e++) {
                const int fe = e == 0 ? f1 : f2;
                int ra[2];
                face_axes(fe, ra[0], ra[1]);
                const float *c0 = e == 0 ? x1 : x2;
                for (int s = 0; s < 2 && !mixed; s++) {
                    const int P = 2 * s, M = 2 * s + 1;
                    const double *scs = sc[s];
                    const float *cp = nullptr, *cm = nullptr;
                    if (has[P] && !(NR->st[nid[P]] & kBad) && (e == 0 ? NR->f1 : NR->f2)[nid[P]] == fe)
                        cp = (e == 0 ? NR->xi1 : NR->xi2) + 3 * nid[P];
                    if (has[M] && !(NR->st[nid[M]] & kBad) && (e == 0 ? NR->f1 : NR->f2)[nid[M]] == fe)
                        cm = (e == 0 ? NR->xi1 : NR->xi2) + 3 * nid[M];
                    for (int r = 0; r < 2; r++) {
                        const int a = ra[r];
                        // (the halving is exact in float: one FP64 multiply per entry)
                        if (cp && cm) Jm[e][r][s] = trace::f2d(0.5f * (cp[a] - cm[a])) * scs[a];
                        else if (cp) Jm[e][r][s] = trace::f2d(cp[a] - c0[a]) * scs[a];
                        else if (cm) Jm[e][r][s] = trace::f2d(c0[a] - cm[a]) * scs[a];
                        else mixed = true;
                    }
                }
            }
            if (mixed) {
                st |= FQSL_LINE_MIXED;
            } else {
                const double adj[2][2] = {{Jm[0][1][1], -Jm[0][0][1]}, {-Jm[0][1][0], Jm[0][0][0]}};
                double norm2 = 0.0;
                for (int r = 0; r < 2; r++)
                    for (int s = 0; s < 2; s++) {
                        const double m = Jm[1][r][0] * adj[0][s] + Jm[1][r][1] * adj[1][s];
                        norm2 += m * m;
                    }
                // |Bn1 Bn2| / Bn0^2 as the product of two float quotients
                // (correctly rounded; Bn0 holds the seed pre-pass's float
                // value, and Bn1, Bn2 are float gathers), widened exactly:
                // relative error below 2^-23, on the FP32 pipe
                const float b0 = bits::narrow_exact(R.bn0[idx]);
                const float q1 = bn_at(f, x1, f1) / b0, q2 = bn_at(f, x2, f2) / b0;
                Q = norm2 * fabs(trace::f2d(q1) * trace::f2d(q2));
            }
        }
        const fqsl_out &o = A.out;
        if (o.Q) o.Q[idx] = Q;
        if (o.Tw || o.length) {
            double tw = NAN, len = NAN;
            if (!bad) {
                const float4 k0 = R.kacc[2 * idx], k1 = R.kacc[2 * idx + 1];
                len = (trace::f2d(k0.x) - trace::f2d(k0.y)) + (trace::f2d(k1.x) - trace::f2d(k1.y));
                tw = (trace::f2d(k0.z) - trace::f2d(k0.w)) + (trace::f2d(k1.z) - trace::f2d(k1.w));
            }
            if (o.Tw) o.Tw[idx] = tw;
            if (o.length) o.length[idx] = len;
        }
        if (o.r1)
            for (int c = 0; c < 3; c++) o.r1[3 * idx + c] = fma(f.d[c], trace::f2d(x1[c]), f.o[c]);
        if (o.r2)
            for (int c = 0; c < 3; c++) o.r2[3 * idx + c] = fma(f.d[c], trace::f2d(x2[c]), f.o[c]);
        if (o.face1) o.face1[idx] = (int8_t)f1;
        if (o.face2) o.face2[idx] = (int8_t)f2;
        if (o.status) o.status[idx] = (uint8_t)st;
        if (o.steps) o.steps[idx] = R.steps[idx];
    }
}

namespace {

// (4 blocks of 256 per SM, 64 registers: the kernel waits on the FP64 pipe and
// on the neighbouring lines' records. On the 1024^2 map: 0.123 ms, against
// 0.141 ms at 3 blocks, 0.137 ms at 5 and 6, and 0.170 ms with the compiler's
// unconstrained 86 registers, which fit only 2)
__global__ void __launch_bounds__(256, 4) k_assemble_f32(const AssembleArgs A)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
         idx += (long long)gridDim.x * blockDim.x)
        assemble_one_f32(A, idx);
}

// Method II from the FP32 tracer's end deviation vectors (Eq. q_scott), in FP64.
__global__ void __launch_bounds__(256) k_assemble_m2_f32(const AssembleArgs A)
{
    const FieldView &f = A.f;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
         idx += (long long)gridDim.x * blockDim.x) {
        const LineRecs &R = A.rec;
        const unsigned st = R.st[idx];
        const bool bad = (st & kBad) != 0;
        const float *x1 = R.xi1 + 3 * idx, *x2 = R.xi2 + 3 * idx;
        const int f1 = R.f1[idx], f2 = R.f2[idx];
        double Q = NAN;
        if (!bad) {
            double Ut[2][3], Vt[2][3], bn[2];
            for (int e = 0; e < 2; e++) {
                const int a = (e == 0 ? f1 : f2) >> 1;
                const float *xe = e == 0 ? x1 : x2;
                float Bf[3], Jf[3];
                if (f.rect) trace::gather_rect(f, xe[0], xe[1], xe[2], Bf, Jf);
                else trace::gather(f, xe[0], xe[1], xe[2], Bf, Jf);
                const double B[3] = {trace::f2d(Bf[0]), trace::f2d(Bf[1]), trace::f2d(Bf[2])};
                const float *dv = R.dev32 + 12 * idx + 6 * e;
                const double U[3] = {trace::f2d(dv[0]), trace::f2d(dv[1]), trace::f2d(dv[2])},
                             V[3] = {trace::f2d(dv[3]), trace::f2d(dv[4]), trace::f2d(dv[5])};
                double ru, rv;
                if (A.qperp) {
                    // Q_perp: the end plane perpendicular to B
                    const double BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
                    bn[e] = sqrt(BB);
                    ru = (U[0] * B[0] + U[1] * B[1] + U[2] * B[2]) / BB;
                    rv = (V[0] * B[0] + V[1] * B[1] + V[2] * B[2]) / BB;
                } else {
                    bn[e] = B[a];
                    ru = U[a] / B[a];
                    rv = V[a] / B[a];
                }
                for (int b = 0; b < 3; b++) {
                    Ut[e][b] = U[b] - ru * B[b];
                    Vt[e][b] = V[b] - rv * B[b];
                }
            }
            auto dot = [](const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
            const double num = dot(Ut[0], Ut[0]) * dot(Vt[1], Vt[1]) + dot(Ut[1], Ut[1]) * dot(Vt[0], Vt[0]) -
                               2.0 * dot(Ut[0], Vt[0]) * dot(Ut[1], Vt[1]);
            const double bn0 = R.bn0[idx];
            Q = fabs(num) * fabs(bn[0] * bn[1]) / (bn0 * bn0);
        }
        const fqsl_out &o = A.out;
        if (o.Q) o.Q[idx] = Q;
        if (o.Tw || o.length) {
            double tw = NAN, len = NAN;
            if (!bad) {
                const float4 k0 = R.kacc[2 * idx], k1 = R.kacc[2 * idx + 1];
                len = (trace::f2d(k0.x) - trace::f2d(k0.y)) + (trace::f2d(k1.x) - trace::f2d(k1.y));
                tw = (trace::f2d(k0.z) - trace::f2d(k0.w)) + (trace::f2d(k1.z) - trace::f2d(k1.w));
            }
            if (o.Tw) o.Tw[idx] = tw;
            if (o.length) o.length[idx] = len;
        }
        if (o.r1)
            for (int c = 0; c < 3; c++) o.r1[3 * idx + c] = fma(f.d[c], trace::f2d(x1[c]), f.o[c]);
        if (o.r2)
            for (int c = 0; c < 3; c++) o.r2[3 * idx + c] = fma(f.d[c], trace::f2d(x2[c]), f.o[c]);
        if (o.face1) o.face1[idx] = (int8_t)f1;
        if (o.face2) o.face2[idx] = (int8_t)f2;
        if (o.status) o.status[idx] = (uint8_t)st;
        if (o.steps) o.steps[idx] = R.steps[idx];
    }
}

}  // namespace

cudaError_t launch_assemble_m2_f32(const AssembleArgs &a, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (a.n + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    k_assemble_m2_f32<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

namespace {
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

__global__ void __launch_bounds__(256, 4) k_batch_assemble_f32(const AssembleArgs *__restrict__ desc,
                                                            const long long *__restrict__ nbase, int nent)
{
    const long long total = nbase[nent];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = batch_entry(nbase, nent, idx);
        assemble_one_f32(desc[b], idx - nbase[b]);
    }
}
}  // namespace

cudaError_t launch_batch_assemble_f32(const AssembleArgs *desc, const long long *nbase, int nent, long long total,
                                      cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    k_batch_assemble_f32<<<(unsigned)blocks, 256, 0, s>>>(desc, nbase, nent);
    return cudaGetLastError();
}

cudaError_t launch_assemble_f32(const AssembleArgs &a, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (a.n + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_assemble_f32<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fqsl
