// curl_pack: curl B at the nodes and the packed B+J node records.
//
// The twist number Tw = int (curl B . B)/(4 pi B^2) dl (Sec. 1, Eq. tw) needs
// curl B along the line; it is precomputed once per field on the node grid
// with 2nd-order central differences inside (the stencil of Eq. grad_B),
// 2nd-order one-sided differences on the faces and first order on a 2-node
// axis, and packed next to B so that one trilinear gather (Sec. 2.2, Eq.
// interp) fetches both. FP64 records (and FP32 records of an FP64 cube) use
// FP64 stencils written as plain expressions; FP32 records of an FP32 cube use
// float stencils. On a stretched grid the three-point stencils of a
// non-uniform axis are used, in FP64. One thread per node, grid-stride;
// streaming and HBM-bound.
#include "fqsl_internal.cuh"

namespace fqsl {
namespace {

template <typename TI>
__device__ __forceinline__ double node_diff(const TI *__restrict__ B, int c, long long node, long long stride,
                                            long long i, long long n, double h)
{
    // value of component c at index kk along the axis (node is at index i)
    auto F = [&](long long kk) -> double { return (double)B[(node + (kk - i) * stride) * 3 + c]; };
    if (n == 2) return (F(1) - F(0)) / h;
    if (i == 0) return (-3.0 * F(0) + 4.0 * F(1) - F(2)) / (2.0 * h);
    if (i == n - 1) return (3.0 * F(n - 1) - 4.0 * F(n - 2) + F(n - 3)) / (2.0 * h);
    return (F(i + 1) - F(i - 1)) / (2.0 * h);
}

template <typename TI>
__global__ void __launch_bounds__(256) k_curl_pack(const TI *__restrict__ B, int nx, int ny, int nz, double dx,
                                                   double dy, double dz, float4 *__restrict__ rec32,
                                                   double2 *__restrict__ rec64)
{
    const long long total = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const long long i = node % nx;
        const long long j = (node / nx) % ny;
        const long long k = node / sz;
        const double dyBz = node_diff(B, 2, node, sy, j, ny, dy);
        const double dzBy = node_diff(B, 1, node, sz, k, nz, dz);
        const double dzBx = node_diff(B, 0, node, sz, k, nz, dz);
        const double dxBz = node_diff(B, 2, node, 1, i, nx, dx);
        const double dxBy = node_diff(B, 1, node, 1, i, nx, dx);
        const double dyBx = node_diff(B, 0, node, sy, j, ny, dy);
        const double Jx = dyBz - dzBy, Jy = dzBx - dxBz, Jz = dxBy - dyBx;
        const double Bx = (double)B[node * 3 + 0], By = (double)B[node * 3 + 1], Bz = (double)B[node * 3 + 2];
        if (rec32) {
            rec32[2 * node + 0] = make_float4((float)Bx, (float)By, (float)Bz, (float)Jx);
            rec32[2 * node + 1] = make_float4((float)Jy, (float)Jz, 0.f, 0.f);
        }
        if (rec64) {
            rec64[4 * node + 0] = make_double2(Bx, By);
            rec64[4 * node + 1] = make_double2(Bz, Jx);
            rec64[4 * node + 2] = make_double2(Jy, Jz);
            rec64[4 * node + 3] = make_double2(0.0, 0.0);
        }
    }
}

// Stretched grid (Sec. 2.2): d f/d x_a at node index i along an axis, as the
// derivative of the quadratic through three neighbouring nodes (one-sided at
// the ends, first order on a 2-node axis); on a uniform axis these are the
// stencils above. co = the node's three coefficients, formed on the host
// from the node coordinates X (fqsl_field_create_rect); with them each
// derivative is a plain sum of products in a fixed order:
//   inside: c0 f_{i-1} + c1 f_i + c2 f_{i+1}; first node: c0 f_0 + c1 f_1 -
//   c2 f_2; last node: c0 f_{n-3} - c1 f_{n-2} + c2 f_{n-1}.
template <typename TI>
__device__ __forceinline__ double node_diff_rect(const TI *__restrict__ B, int c, long long node, long long stride,
                                                 long long i, long long n, const double *__restrict__ X,
                                                 const double *__restrict__ co)
{
    auto F = [&](long long kk) -> double { return (double)B[(node + (kk - i) * stride) * 3 + c]; };
    if (n == 2) return (F(1) - F(0)) / (X[1] - X[0]);
    const double c0 = co[3 * i], c1 = co[3 * i + 1], c2 = co[3 * i + 2];
    if (i == 0) return c0 * F(0) + c1 * F(1) - c2 * F(2);
    if (i == n - 1) return c0 * F(n - 3) - c1 * F(n - 2) + c2 * F(n - 1);
    return c0 * F(i - 1) + c1 * F(i) + c2 * F(i + 1);
}

template <typename TI>
__global__ void __launch_bounds__(256) k_curl_pack_rect(const TI *__restrict__ B, const FieldView g,
                                                        float4 *__restrict__ rec32, double2 *__restrict__ rec64)
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long total = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const long long i = node % nx;
        const long long j = (node / nx) % ny;
        const long long k = node / sz;
        const double dyBz = node_diff_rect(B, 2, node, sy, j, ny, g.x64[1], g.dco[1]);
        const double dzBy = node_diff_rect(B, 1, node, sz, k, nz, g.x64[2], g.dco[2]);
        const double dzBx = node_diff_rect(B, 0, node, sz, k, nz, g.x64[2], g.dco[2]);
        const double dxBz = node_diff_rect(B, 2, node, 1, i, nx, g.x64[0], g.dco[0]);
        const double dxBy = node_diff_rect(B, 1, node, 1, i, nx, g.x64[0], g.dco[0]);
        const double dyBx = node_diff_rect(B, 0, node, sy, j, ny, g.x64[1], g.dco[1]);
        const double Jx = dyBz - dzBy, Jy = dzBx - dxBz, Jz = dxBy - dyBx;
        const double Bx = (double)B[node * 3 + 0], By = (double)B[node * 3 + 1], Bz = (double)B[node * 3 + 2];
        if (rec32) {
            rec32[2 * node + 0] = make_float4((float)Bx, (float)By, (float)Bz, (float)Jx);
            rec32[2 * node + 1] = make_float4((float)Jy, (float)Jz, 0.f, 0.f);
        }
        if (rec64) {
            rec64[4 * node + 0] = make_double2(Bx, By);
            rec64[4 * node + 1] = make_double2(Bz, Jx);
            rec64[4 * node + 2] = make_double2(Jy, Jz);
            rec64[4 * node + 3] = make_double2(0.0, 0.0);
        }
    }
}

// FP32 records only: the same stencils in float with reciprocal spacings (the
// FP64 kernel above is the one whose rounding matches a plain evaluation).
__device__ __forceinline__ float node_diff32(const float *__restrict__ B, int c, unsigned node, unsigned stride,
                                             unsigned i, unsigned n, float rh, float rh2)
{
    auto F = [&](unsigned kk) -> float { return B[(size_t)(node + kk * stride - i * stride) * 3 + c]; };
    if (n == 2) return (F(1) - F(0)) * rh;
    if (i == 0) return (-3.f * F(0) + 4.f * F(1) - F(2)) * rh2;
    if (i == n - 1) return (3.f * F(n - 1) - 4.f * F(n - 2) + F(n - 3)) * rh2;
    return (F(i + 1) - F(i - 1)) * rh2;
}

// 32-bit index arithmetic (a cube with FP32 records holds fewer than 2^31 nodes)
__global__ void __launch_bounds__(256) k_curl_pack32(const float *__restrict__ B, int nx, int ny, int nz, float rx,
                                                     float ry, float rz, float4 *__restrict__ rec32)
{
    const unsigned total = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    const unsigned sy = (unsigned)nx, sz = (unsigned)nx * (unsigned)ny;
    for (unsigned node = blockIdx.x * blockDim.x + threadIdx.x; node < total; node += gridDim.x * blockDim.x) {
        const unsigned t = node / sy;
        const unsigned i = node - t * sy;
        const unsigned k = t / (unsigned)ny;
        const unsigned j = t - k * (unsigned)ny;
        const float dyBz = node_diff32(B, 2, node, sy, j, ny, ry, 0.5f * ry);
        const float dzBy = node_diff32(B, 1, node, sz, k, nz, rz, 0.5f * rz);
        const float dzBx = node_diff32(B, 0, node, sz, k, nz, rz, 0.5f * rz);
        const float dxBz = node_diff32(B, 2, node, 1, i, nx, rx, 0.5f * rx);
        const float dxBy = node_diff32(B, 1, node, 1, i, nx, rx, 0.5f * rx);
        const float dyBx = node_diff32(B, 0, node, sy, j, ny, ry, 0.5f * ry);
        rec32[2 * (size_t)node + 0] = make_float4(B[(size_t)node * 3 + 0], B[(size_t)node * 3 + 1], B[(size_t)node * 3 + 2], dyBz - dzBy);
        rec32[2 * (size_t)node + 1] = make_float4(dzBx - dxBz, dxBy - dyBx, 0.f, 0.f);
    }
}

// Component c of B/|B| at a node (0 where |B| = 0), as written.
template <typename TI>
__device__ __forceinline__ double bhat(const TI *__restrict__ B, long long q, int c)
{
    const double b0 = (double)B[3 * q], b1 = (double)B[3 * q + 1], b2 = (double)B[3 * q + 2];
    const double m = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
    const double bc = c == 0 ? b0 : (c == 1 ? b1 : b2);
    return m > 0 ? bc / m : 0.0;
}

template <typename TI>
__device__ __forceinline__ double bhat_diff(const TI *__restrict__ B, int c, long long node, long long stride,
                                            long long i, long long n, double h)
{
    auto F = [&](long long kk) -> double { return bhat(B, node + (kk - i) * stride, c); };
    if (n == 2) return (F(1) - F(0)) / h;
    if (i == 0) return (-3.0 * F(0) + 4.0 * F(1) - F(2)) / (2.0 * h);
    if (i == n - 1) return (3.0 * F(n - 1) - 4.0 * F(n - 2) + F(n - 3)) / (2.0 * h);
    return (F(i + 1) - F(i - 1)) / (2.0 * h);
}

// Stretched grid: the same with the three-point stencils of node_diff_rect
template <typename TI>
__device__ __forceinline__ double bhat_diff_rect(const TI *__restrict__ B, int c, long long node, long long stride,
                                                 long long i, long long n, const double *__restrict__ X,
                                                 const double *__restrict__ co)
{
    auto F = [&](long long kk) -> double { return bhat(B, node + (kk - i) * stride, c); };
    if (n == 2) return (F(1) - F(0)) / (X[1] - X[0]);
    const double c0 = co[3 * i], c1 = co[3 * i + 1], c2 = co[3 * i + 2];
    if (i == 0) return c0 * F(0) + c1 * F(1) - c2 * F(2);
    if (i == n - 1) return c0 * F(n - 3) - c1 * F(n - 2) + c2 * F(n - 1);
    return c0 * F(i - 1) + c1 * F(i) + c2 * F(i + 1);
}

template <typename TI>
__global__ void __launch_bounds__(256) k_gradb_pack_rect(const TI *__restrict__ B, const FieldView g,
                                                         float *__restrict__ g32, double *__restrict__ g64)
{
    const long long nx = g.nx, ny = g.ny, nz = g.nz;
    const long long total = nx * ny * nz;
    const long long stride[3] = {1, nx, nx * ny};
    const long long n[3] = {nx, ny, nz};
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const long long idx[3] = {node % nx, (node / nx) % ny, node / stride[2]};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                const double v = bhat_diff_rect(B, b, node, stride[a], idx[a], n[a], g.x64[a], g.dco[a]);
                if (g64) g64[node * 10 + a * 3 + b] = v;
                if (g32) g32[node * 12 + a * 3 + b] = (float)v;
            }
        if (g64) g64[node * 10 + 9] = 0.0;
        if (g32) g32[node * 12 + 9] = g32[node * 12 + 10] = g32[node * 12 + 11] = 0.f;
    }
}

// grad(B/|B|) at the nodes for Method II way 1 (Sec. 4, Eq. grad_B): G[a*3+b]
// = d(B_b/|B|)/dx_a with the stencils of the curl grid.
template <typename TI>
__global__ void __launch_bounds__(256) k_gradb_pack(const TI *__restrict__ B, int nx, int ny, int nz, double dx,
                                                    double dy, double dz, float *__restrict__ g32,
                                                    double *__restrict__ g64)
{
    const long long total = (long long)nx * ny * nz;
    const long long stride[3] = {1, nx, (long long)nx * ny};
    const double d[3] = {dx, dy, dz};
    const long long n[3] = {nx, ny, nz};
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < total;
         node += (long long)gridDim.x * blockDim.x) {
        const long long idx[3] = {node % nx, (node / nx) % ny, node / stride[2]};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                const double g = bhat_diff(B, b, node, stride[a], idx[a], n[a], d[a]);
                if (g64) g64[node * 10 + a * 3 + b] = g;
                if (g32) g32[node * 12 + a * 3 + b] = (float)g;
            }
        if (g64) g64[node * 10 + 9] = 0.0;
        if (g32) g32[node * 12 + 9] = g32[node * 12 + 10] = g32[node * 12 + 11] = 0.f;
    }
}

}  // namespace

cudaError_t launch_gradb_pack(const void *B, fqsl_dtype bt, const FieldView &g, void *grad32, void *grad64,
                              cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)g.nx * g.ny * g.nz;
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    if (g.rect) {
        if (bt == FQSL_F32)
            k_gradb_pack_rect<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)B, g, (float *)grad32,
                                                                     (double *)grad64);
        else
            k_gradb_pack_rect<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)B, g, (float *)grad32,
                                                                      (double *)grad64);
        return cudaGetLastError();
    }
    if (bt == FQSL_F32)
        k_gradb_pack<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)B, g.nx, g.ny, g.nz, g.d[0], g.d[1],
                                                            g.d[2], (float *)grad32, (double *)grad64);
    else
        k_gradb_pack<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)B, g.nx, g.ny, g.nz, g.d[0], g.d[1],
                                                             g.d[2], (float *)grad32, (double *)grad64);
    return cudaGetLastError();
}

cudaError_t launch_curl_pack(const void *B, fqsl_dtype bt, const FieldView &g, void *rec32, void *rec64,
                             cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)g.nx * g.ny * g.nz;
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (g.rect) {
        // stretched grid: FP64 stencils for every record precision
        if (bt == FQSL_F32)
            k_curl_pack_rect<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)B, g, (float4 *)rec32,
                                                                    (double2 *)rec64);
        else
            k_curl_pack_rect<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)B, g, (float4 *)rec32,
                                                                     (double2 *)rec64);
        return cudaGetLastError();
    }
    if (bt == FQSL_F32 && rec32) {
        // FP32 records from an FP32 cube: float stencils (the FP64 records, if
        // also wanted, come from the FP64 stencils below)
        k_curl_pack32<<<(unsigned)blocks, 256, 0, s>>>((const float *)B, g.nx, g.ny, g.nz, (float)(1.0 / g.d[0]),
                                                       (float)(1.0 / g.d[1]), (float)(1.0 / g.d[2]),
                                                       (float4 *)rec32);
        if (rec64)
            k_curl_pack<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)B, g.nx, g.ny, g.nz, g.d[0], g.d[1],
                                                               g.d[2], nullptr, (double2 *)rec64);
    } else if (bt == FQSL_F32)
        k_curl_pack<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)B, g.nx, g.ny, g.nz, g.d[0], g.d[1],
                                                           g.d[2], (float4 *)rec32, (double2 *)rec64);
    else
        k_curl_pack<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)B, g.nx, g.ny, g.nz, g.d[0], g.d[1],
                                                            g.d[2], (float4 *)rec32, (double2 *)rec64);
    return cudaGetLastError();
}

}  // namespace fqsl
