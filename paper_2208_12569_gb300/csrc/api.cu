// C ABI of the fqsl library (declared in include/fqsl.h): argument checks,
// handle and scratch management, and the launch sequence of each call.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "fqsl_internal.cuh"

using namespace fqsl;

namespace {

thread_local std::string g_err;

fqsl_status fail(fqsl_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

fqsl_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(FQSL_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FQSL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Every device allocation of the library goes through dev_malloc, so that a
// test can make one fail as out of memory on demand (fqsl_debug_alloc_cap):
// the failure paths run without exhausting the GPU.
std::atomic<unsigned long long> g_alloc_cap{0};

cudaError_t dev_malloc(void **p, size_t bytes)
{
    const unsigned long long cap = g_alloc_cap.load();
    if (cap != 0 && (unsigned long long)bytes > cap) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

bool finite3(const double *v) { return v && isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// 1 <= a, 1 <= b and a * b <= lim, decided without forming a product that can
// overflow
bool count_ok(long long a, long long b, long long lim) { return a >= 1 && b >= 1 && a <= lim && b <= lim / a; }

constexpr long long kMaxCount = (1LL << 31) - 1;  // largest number of seeds (or nodes) of one call

// sequential carve of one scratch allocation
struct Carver {
    char *base;
    size_t off = 0;
    template <typename P>
    P *take(size_t count)
    {
        P *p = base ? (P *)(base + off) : nullptr;
        off = align_up(off + count * sizeof(P));
        return p;
    }
};

}  // namespace

struct fqsl_field_s {
    int device = 0;
    int sms = 0;
    FieldView g{};
    void *rec32 = nullptr, *rec64 = nullptr;
    void *grad32 = nullptr, *grad64 = nullptr;  // Method II way 1 gradient grid
    void *scratch = nullptr;
    size_t scratch_cap = 0;
    void *rect_buf = nullptr;  // stretched grid: coordinate, width and bucket tables (FieldView::x64 ...)
    unsigned long long *counters = nullptr;  // [0] primary head, [1] extra head, [2] rotated count (low 32 bits),
                                             // [4] first failed index check of the adjoint kernels, [5] their count
    int blocks_cache[2][3][3] = {};  // [scheme][precision][source] resident blocks per SM
    int blocks_cache_m2[2][2][2] = {};  // Method II: [scheme][fp64][way - 1]
    int blocks_cache_tape[2][3][2] = {};  // taped tracers: [scheme][precision][lattice, extra]
    bool timing = false, timed = false, extra_timed = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned long long serial = 0;  // unique per handle made in this process (tapes name their field by it)
    unsigned long long gen = 0;     // incremented by every fqsl_field_update
    std::mutex mu;
};

// A taped plane or volume map (for fqsl_backward): its line records, step
// tape and adjoint buffers live in buf, the reverse sweep's per-step arrays in
// work. The tape names the field it was recorded on by handle and serial, and
// the field's record generation at that time.
struct fqsl_tape_s {
    bool valid = false;
    fqsl_field field = nullptr;
    unsigned long long field_serial = 0;
    unsigned long long gen = 0;
    Lattice lat{};
    fqsl_params p{};
    bool face_plane = false;
    size_t nodes = 0;      // the field's node count (size of the adjoint node grid)
    long long pool = 0;    // tape chunks of the next taped call
    long long keep_cap = 0;   // chunks whose states the taped call keeps (Tape::wcap; 0: first guess)
    long long keep_want = 0;  // what the last backward call needed (applied at the next taped call)
    void *buf = nullptr;
    size_t cap = 0;
    void *work = nullptr;  // per-step arrays of the reverse sweep
    size_t work_cap = 0;
    // the chunks the last taped call used, copied to pinned host memory as
    // soon as its tracers finish (used_ev), so that fqsl_backward waits for
    // the tracers only, not for what the stream runs after them
    unsigned long long *used_host = nullptr;
    cudaEvent_t used_ev = nullptr;
};

namespace {
std::atomic<unsigned long long> g_field_serial{0};

void mark(fqsl_field f, int i, cudaStream_t s)
{
    if (f->timing) cudaEventRecord(f->ev[i], s);
}

// argument checks shared by the two field constructors
fqsl_status check_create(const void *B_dev, fqsl_dtype b_dtype, long long nx, long long ny, long long nz,
                         unsigned flags, fqsl_field *out, const char *who)
{
    if (!out) return fail(FQSL_ERR_ARG, "%s: out is NULL", who);
    if (!B_dev) return fail(FQSL_ERR_ARG, "%s: B_dev is NULL", who);
    if (b_dtype != FQSL_F32 && b_dtype != FQSL_F64)
        return fail(FQSL_ERR_ARG, "%s: b_dtype must be FQSL_F32 or FQSL_F64", who);
    if (nx < 2 || ny < 2 || nz < 2) return fail(FQSL_ERR_ARG, "%s: need nx, ny, nz >= 2", who);
    if (nx >= (1 << 23) || ny >= (1 << 23) || nz >= (1 << 23) || !count_ok(nx * ny, nz, kMaxCount))
        return fail(FQSL_ERR_ARG, "%s: grid too large (each axis < 2^23 nodes, < 2^31 nodes)", who);
    if (!(flags & (FQSL_PACK_F32 | FQSL_PACK_F64)) || (flags & ~(FQSL_PACK_F32 | FQSL_PACK_F64 | FQSL_PACK_GRADB)))
        return fail(FQSL_ERR_ARG, "%s: flags must hold FQSL_PACK_F32 and/or FQSL_PACK_F64 "
                                  "(and optionally FQSL_PACK_GRADB)", who);
    if (((uintptr_t)B_dev) % 16) return fail(FQSL_ERR_ARG, "%s: B_dev must be 16-byte aligned", who);
    return FQSL_OK;
}

// B_dev must be device (or managed) memory; checked after the host-side
// argument checks
fqsl_status check_device_ptr(const void *B_dev, const char *who)
{
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, B_dev);
    if (e != cudaSuccess || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(FQSL_ERR_ARG, "%s: B_dev is not device memory", who);
    }
    return FQSL_OK;
}

void set_dims(fqsl_field f, long long nx, long long ny, long long nz)
{
    f->serial = ++g_field_serial;
    cudaGetDevice(&f->device);
    cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, f->device);
    f->g.nx = (int)nx;
    f->g.ny = (int)ny;
    f->g.nz = (int)nz;
    f->g.cmax[0] = (float)(nx - 2);
    f->g.cmax[1] = (float)(ny - 2);
    f->g.cmax[2] = (float)(nz - 2);
    f->g.sy32 = (unsigned)(nx * 32);
    f->g.sz32 = (unsigned)(nx * ny * 32 <= 0xffffffffLL ? nx * ny * 32 : 0);
    f->g.nodes = nx * ny * nz;
    f->g.err = nullptr;
}

// release everything a handle under construction may hold
void free_field(fqsl_field f)
{
    cudaFree(f->rec32);
    cudaFree(f->rec64);
    cudaFree(f->grad32);
    cudaFree(f->grad64);
    cudaFree(f->counters);
    cudaFree(f->rect_buf);
    delete f;
}

// records, counters and the first packing of a handle whose geometry is set
fqsl_status finish_create(fqsl_field f, const void *B_dev, fqsl_dtype b_dtype, unsigned flags, void *cuda_stream,
                          fqsl_field *out, const char *who)
{
    const size_t nodes = (size_t)f->g.nodes;
    cudaError_t e = cudaSuccess;
    if (flags & FQSL_PACK_F32) e = dev_malloc((void **)&f->rec32, nodes * 32);
    if (e == cudaSuccess && (flags & FQSL_PACK_F64)) e = dev_malloc((void **)&f->rec64, nodes * 64);
    if (e == cudaSuccess && (flags & FQSL_PACK_GRADB)) {
        if (f->rec32) e = dev_malloc((void **)&f->grad32, nodes * 48);
        if (e == cudaSuccess && f->rec64) e = dev_malloc((void **)&f->grad64, nodes * 80);
    }
    if (e == cudaSuccess) e = dev_malloc((void **)&f->counters, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_field(f);
        return cuda_fail(e, who);
    }
    e = cudaMemsetAsync(f->counters, 0, 8 * sizeof(unsigned long long), (cudaStream_t)cuda_stream);
    if (e == cudaSuccess) e = launch_curl_pack(B_dev, b_dtype, f->g, f->rec32, f->rec64, (cudaStream_t)cuda_stream);
    if (e == cudaSuccess && (f->grad32 || f->grad64))
        e = launch_gradb_pack(B_dev, b_dtype, f->g, f->grad32, f->grad64, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        free_field(f);
        return cuda_fail(e, who);
    }
    *out = f;
    return FQSL_OK;
}
}  // namespace

extern "C" {

void fqsl_params_default(fqsl_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->method = 1;
    p->gradb_way = 1;
    p->precision = FQSL_F32;
    p->tol = pow(10.0, -3.2);
    p->h0 = 0.5;
    p->h_min = 1e-6;
    p->h_max = 4.0;
    p->max_steps = 100000;
    p->rot_thresh = 0.05;
    p->tol_exp = 1.5;
    p->graze = 1e-3;
    p->eps_way2 = 1e-3;
    p->sync_dirs = -1;
    p->reverse_precision = -1;
    p->scheme = 0;
    p->step = 3.0;
    p->step_min = 0.15;
}

const char *fqsl_version(void) { return "fqsl 0.1.0 (sm_103a)"; }

void fqsl_debug_alloc_cap(unsigned long long bytes) { g_alloc_cap.store(bytes); }

const char *fqsl_last_error(void) { return g_err.c_str(); }

fqsl_status fqsl_field_create(const void *B_dev, fqsl_dtype b_dtype, long long nx, long long ny, long long nz,
                              const double origin[3], const double spacing[3], unsigned flags, void *cuda_stream,
                              fqsl_field *out)
{
    g_err.clear();
    const char *who = "fqsl_field_create";
    if (out) *out = nullptr;
    fqsl_status st = check_create(B_dev, b_dtype, nx, ny, nz, flags, out, who);
    if (st != FQSL_OK) return st;
    if (!finite3(origin) || !finite3(spacing)) return fail(FQSL_ERR_ARG, "%s: origin/spacing must be finite", who);
    if (!(spacing[0] > 0 && spacing[1] > 0 && spacing[2] > 0))
        return fail(FQSL_ERR_ARG, "%s: spacing must be > 0", who);
    st = check_device_ptr(B_dev, who);
    if (st != FQSL_OK) return st;
    fqsl_field f = new (std::nothrow) fqsl_field_s();
    if (!f) return fail(FQSL_ERR_OOM, "%s: host allocation failed", who);
    set_dims(f, nx, ny, nz);
    for (int a = 0; a < 3; a++) {
        f->g.o[a] = origin[a];
        f->g.d[a] = spacing[a];
        f->g.rd[a] = (float)(1.0 / spacing[a]);
    }
    f->g.unit = spacing[0] == 1.0 && spacing[1] == 1.0 && spacing[2] == 1.0;
    return finish_create(f, B_dev, b_dtype, flags, cuda_stream, out, who);
}

fqsl_status fqsl_field_create_rect(const void *B_dev, fqsl_dtype b_dtype, long long nx, long long ny, long long nz,
                                   const double *x, const double *y, const double *z, unsigned flags,
                                   void *cuda_stream, fqsl_field *out)
{
    g_err.clear();
    const char *who = "fqsl_field_create_rect";
    if (out) *out = nullptr;
    fqsl_status st = check_create(B_dev, b_dtype, nx, ny, nz, flags, out, who);
    if (st != FQSL_OK) return st;
    const double *X[3] = {x, y, z};
    const long long N[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++) {
        if (!X[a]) return fail(FQSL_ERR_ARG, "%s: coordinate array %d is NULL", who, a);
        for (long long i = 0; i < N[a]; i++)
            if (!isfinite(X[a][i])) return fail(FQSL_ERR_ARG, "%s: coordinate %d of axis %d is not finite", who, (int)i, a);
        for (long long i = 0; i + 1 < N[a]; i++)
            if (!(X[a][i + 1] > X[a][i]))
                return fail(FQSL_ERR_ARG, "%s: axis %d coordinates are not strictly increasing at %lld", who, a, i);
        if (flags & FQSL_PACK_F32)
            for (long long i = 0; i + 1 < N[a]; i++)
                if (!((float)(X[a][i + 1] - X[a][0]) > (float)(X[a][i] - X[a][0])))
                    return fail(FQSL_ERR_ARG, "%s: axis %d cells %lld, %lld collapse in float (FP32 records)", who,
                                a, i, i + 1);
    }
    st = check_device_ptr(B_dev, who);
    if (st != FQSL_OK) return st;
    // host tables, one device buffer: x64 | cell64 | cell32 | bkt | bk32 | dco
    std::vector<double> x64, dco;
    std::vector<double2> cell64;
    std::vector<float4> cell32;
    std::vector<int> bkt;
    std::vector<float4> bk32;
    long long nb[3];
    float hi32[3];
    for (int a = 0; a < 3; a++) {
        const double *A = X[a];
        const long long n = N[a];
        const double L = A[n - 1] - A[0];
        double wmin = INFINITY;
        for (long long i = 0; i + 1 < n; i++) wmin = fmin(wmin, A[i + 1] - A[i]);
        // buckets no wider than the narrowest cell, within [n - 1, 16 (n - 1)] and below 2^22
        long long b = (long long)ceil(L / wmin);
        if (b < n - 1) b = n - 1;
        if (b > 16 * (n - 1)) b = 16 * (n - 1);
        if (b > (1LL << 22)) b = 1LL << 22;
        nb[a] = b;
        std::vector<float> r(n);
        for (long long i = 0; i < n; i++) {
            x64.push_back(A[i]);
            r[i] = (float)(A[i] - A[0]);
            // curl stencil coefficients of node i: the derivative of the
            // quadratic through three neighbouring nodes (see field.cu)
            double c0 = 0.0, c1 = 0.0, c2 = 0.0;
            if (n > 2) {
                if (i == 0) {
                    const double h1 = A[1] - A[0], h2 = A[2] - A[1];
                    c0 = -(2.0 * h1 + h2) / (h1 * (h1 + h2));
                    c1 = (h1 + h2) / (h1 * h2);
                    c2 = h1 / (h2 * (h1 + h2));
                } else if (i == n - 1) {
                    const double h1 = A[n - 2] - A[n - 3], h2 = A[n - 1] - A[n - 2];
                    c0 = h2 / (h1 * (h1 + h2));
                    c1 = (h1 + h2) / (h1 * h2);
                    c2 = (h1 + 2.0 * h2) / (h2 * (h1 + h2));
                } else {
                    const double h1 = A[i] - A[i - 1], h2 = A[i + 1] - A[i];
                    c0 = -h2 / (h1 * (h1 + h2));
                    c1 = (h2 - h1) / (h1 * h2);
                    c2 = h1 / (h2 * (h1 + h2));
                }
            }
            dco.push_back(c0);
            dco.push_back(c1);
            dco.push_back(c2);
        }
        hi32[a] = r[n - 1];
        for (long long i = 0; i + 1 < n; i++) {
            cell64.push_back(make_double2(A[i], A[i + 1]));
            cell32.push_back(make_float4(r[i], r[i + 1], (float)(1.0 / ((double)r[i + 1] - (double)r[i])), 0.f));
        }
        for (long long k = 0; k < b; k++) {
            // the cell of the bucket's lower end (largest i in [0, n-2] with A[i] <= t)
            const double t = A[0] + (double)k * (L / (double)b);
            long long lo = 0, hi = n - 2;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) / 2;
                if (A[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            bkt.push_back((int)lo);
            const int c = (int)lo;
            float cbits;
            memcpy(&cbits, &c, sizeof cbits);
            const float4 c0 = cell32[cell32.size() - (size_t)(n - 1) + (size_t)c];
            const bool last = lo == n - 2;
            const float4 c1 = last ? make_float4(0.f, INFINITY, 0.f, 0.f) : cell32[cell32.size() - (size_t)(n - 1) + (size_t)c + 1];
            bk32.push_back(make_float4(cbits, c0.x, c0.y, c0.z));
            bk32.push_back(make_float4(last ? INFINITY : c0.y, c1.y, c1.z, 0.f));
        }
    }
    fqsl_field f = new (std::nothrow) fqsl_field_s();
    if (!f) return fail(FQSL_ERR_OOM, "%s: host allocation failed", who);
    set_dims(f, nx, ny, nz);
    const size_t s0 = align_up(x64.size() * sizeof(double)), s1 = align_up(cell64.size() * sizeof(double2)),
                 s2 = align_up(cell32.size() * sizeof(float4)), s3 = align_up(bkt.size() * sizeof(int)),
                 s4 = align_up(bk32.size() * sizeof(float4)), s5 = align_up(dco.size() * sizeof(double));
    cudaError_t e = dev_malloc((void **)&f->rect_buf, s0 + s1 + s2 + s3 + s4 + s5);
    if (e != cudaSuccess) {
        delete f;
        cudaGetLastError();
        return cuda_fail(e, "fqsl_field_create_rect: coordinate tables");
    }
    char *base = (char *)f->rect_buf;
    const void *src[6] = {x64.data(), cell64.data(), cell32.data(), bkt.data(), bk32.data(), dco.data()};
    const size_t len[6] = {x64.size() * sizeof(double), cell64.size() * sizeof(double2),
                           cell32.size() * sizeof(float4), bkt.size() * sizeof(int), bk32.size() * sizeof(float4),
                           dco.size() * sizeof(double)};
    const size_t off[6] = {0, s0, s0 + s1, s0 + s1 + s2, s0 + s1 + s2 + s3, s0 + s1 + s2 + s3 + s4};
    for (int k = 0; k < 6 && e == cudaSuccess; k++) e = cudaMemcpy(base + off[k], src[k], len[k], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(f->rect_buf);
        delete f;
        return cuda_fail(e, "fqsl_field_create_rect: coordinate tables");
    }
    FieldView &g = f->g;
    g.rect = 1;
    long long on = 0, oc = 0, ob = 0;
    for (int a = 0; a < 3; a++) {
        const long long n = N[a];
        g.x64[a] = (const double *)(base + off[0]) + on;
        g.dco[a] = (const double *)(base + off[5]) + 3 * on;
        g.cell64[a] = (const double2 *)(base + off[1]) + oc;
        g.cell32[a] = (const float4 *)(base + off[2]) + oc;
        g.bkt[a] = (const int *)(base + off[3]) + ob;
        g.bk32[a] = (const float4 *)(base + off[4]) + 2 * ob;
        g.nbkt[a] = (int)nb[a];
        const double L = X[a][n - 1] - X[a][0];
        g.bsc64[a] = (double)nb[a] / L;
        g.bsc32[a] = (float)g.bsc64[a];
        g.lo64[a] = X[a][0];
        g.hi64[a] = X[a][n - 1];
        g.hi32[a] = hi32[a];
        // FP32 state = physical position relative to the first node
        g.o[a] = X[a][0];
        g.d[a] = 1.0;
        g.rd[a] = 1.f;
        on += n;
        oc += n - 1;
        ob += nb[a];
    }
    return finish_create(f, B_dev, b_dtype, flags, cuda_stream, out, who);
}

fqsl_status fqsl_field_update(fqsl_field f, const void *B_dev, fqsl_dtype b_dtype, void *cuda_stream)
{
    g_err.clear();
    if (!f) return fail(FQSL_ERR_ARG, "fqsl_field_update: NULL handle");
    if (!B_dev) return fail(FQSL_ERR_ARG, "fqsl_field_update: B_dev is NULL");
    if (b_dtype != FQSL_F32 && b_dtype != FQSL_F64)
        return fail(FQSL_ERR_ARG, "fqsl_field_update: b_dtype must be FQSL_F32 or FQSL_F64");
    if (((uintptr_t)B_dev) % 16) return fail(FQSL_ERR_ARG, "fqsl_field_update: B_dev must be 16-byte aligned");
    std::lock_guard<std::mutex> lock(f->mu);
    cudaError_t e = launch_curl_pack(B_dev, b_dtype, f->g, f->rec32, f->rec64, (cudaStream_t)cuda_stream);
    if (e == cudaSuccess && (f->grad32 || f->grad64))
        e = launch_gradb_pack(B_dev, b_dtype, f->g, f->grad32, f->grad64, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "fqsl_field_update: curl_pack launch");
    f->gen++;
    return FQSL_OK;
}

fqsl_status fqsl_field_set_timing(fqsl_field f, int enable)
{
    g_err.clear();
    if (!f) return fail(FQSL_ERR_ARG, "fqsl_field_set_timing: NULL handle");
    std::lock_guard<std::mutex> lock(f->mu);
    if (enable && !f->ev[0]) {
        for (int i = 0; i < 4; i++) {
            cudaError_t e = cudaEventCreate(&f->ev[i]);
            if (e != cudaSuccess) return cuda_fail(e, "fqsl_field_set_timing");
        }
    }
    f->timing = enable != 0;
    f->timed = false;
    return FQSL_OK;
}

fqsl_status fqsl_field_times(fqsl_field f, float ms[3])
{
    g_err.clear();
    if (!f || !ms) return fail(FQSL_ERR_ARG, "fqsl_field_times: NULL argument");
    std::lock_guard<std::mutex> lock(f->mu);
    if (!f->timed) return fail(FQSL_ERR_ARG, "fqsl_field_times: no timed call yet");
    cudaError_t e = cudaEventSynchronize(f->ev[3]);
    if (e != cudaSuccess) return cuda_fail(e, "fqsl_field_times");
    ms[0] = ms[1] = ms[2] = 0.f;
    cudaEventElapsedTime(&ms[0], f->ev[0], f->ev[1]);
    if (f->extra_timed) cudaEventElapsedTime(&ms[1], f->ev[1], f->ev[2]);
    cudaEventElapsedTime(&ms[2], f->ev[2], f->ev[3]);
    return FQSL_OK;
}

fqsl_status fqsl_field_destroy(fqsl_field f)
{
    g_err.clear();
    if (!f) return fail(FQSL_ERR_ARG, "fqsl_field_destroy: NULL handle");
    cudaDeviceSynchronize();
    for (int i = 0; i < 4; i++)
        if (f->ev[i]) cudaEventDestroy(f->ev[i]);
    cudaFree(f->rec32);
    cudaFree(f->rec64);
    cudaFree(f->grad32);
    cudaFree(f->grad64);
    cudaFree(f->scratch);
    cudaFree(f->counters);
    cudaFree(f->rect_buf);
    delete f;
    return FQSL_OK;
}

}  // extern "C"

namespace {

fqsl_status check_params(const fqsl_field f, const fqsl_params *p, const char *who)
{
    if (!f) return fail(FQSL_ERR_ARG, "%s: NULL field", who);
    if (!p) return fail(FQSL_ERR_ARG, "%s: NULL params", who);
    if (p->method != 1 && p->method != 2) return fail(FQSL_ERR_ARG, "%s: method must be 1 or 2", who);
    if (p->gradb_way != 1 && p->gradb_way != 2) return fail(FQSL_ERR_ARG, "%s: gradb_way must be 1 or 2", who);
    if (p->precision != FQSL_F32 && p->precision != FQSL_F64 && p->precision != FQSL_F32_ACC64)
        return fail(FQSL_ERR_ARG, "%s: precision must be FQSL_F32, FQSL_F64 or FQSL_F32_ACC64", who);
    if (!(p->tol > 0) || !isfinite(p->tol)) return fail(FQSL_ERR_ARG, "%s: tol must be > 0", who);
    if (!(p->h_min > 0) || !(p->h_max >= p->h_min) || !(p->h0 >= p->h_min) || !(p->h0 <= p->h_max) ||
        !isfinite(p->h_max))
        return fail(FQSL_ERR_ARG, "%s: need 0 < h_min <= h0 <= h_max", who);
    if (p->max_steps < 1 || p->max_steps > 2000000000LL)
        return fail(FQSL_ERR_ARG, "%s: max_steps must be in [1, 2e9]", who);
    if (!(p->rot_thresh >= 0) || !(p->rot_thresh < 1)) return fail(FQSL_ERR_ARG, "%s: rot_thresh in [0,1)", who);
    if (!(p->tol_exp >= 0) || !isfinite(p->tol_exp)) return fail(FQSL_ERR_ARG, "%s: tol_exp >= 0", who);
    if (!(p->graze > 0) || !(p->graze < 1)) return fail(FQSL_ERR_ARG, "%s: graze in (0,1)", who);
    if (!(p->eps_way2 > 0) || !(p->eps_way2 < 0.5)) return fail(FQSL_ERR_ARG, "%s: eps_way2 in (0,0.5)", who);
    if (p->refill_lanes < 0 || p->refill_lanes > 32) return fail(FQSL_ERR_ARG, "%s: refill_lanes in [0, 32]", who);
    if (p->sync_dirs < -1 || p->sync_dirs > 1) return fail(FQSL_ERR_ARG, "%s: sync_dirs in {-1, 0, 1}", who);
    if (p->chunk_tiles < 0 || p->chunk_tiles > 64) return fail(FQSL_ERR_ARG, "%s: chunk_tiles in [0, 64]", who);
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 64) return fail(FQSL_ERR_ARG, "%s: blocks_per_sm in [0, 64]", who);
    if (p->tape != 0 && p->tape != 1) return fail(FQSL_ERR_ARG, "%s: tape must be 0 or 1", who);
    if (p->tape_chunk < 0 || p->tape_chunk > 32) return fail(FQSL_ERR_ARG, "%s: tape_chunk in [0, 32]", who);
    if (p->reverse_precision < -1 || p->reverse_precision > FQSL_F32_ACC64)
        return fail(FQSL_ERR_ARG, "%s: reverse_precision must be -1, FQSL_F32, FQSL_F64 or FQSL_F32_ACC64", who);
    if (p->tape) {
        const int rp = p->reverse_precision < 0 ? p->precision : p->reverse_precision;
        if (rp == FQSL_F64 ? !f->rec64 : !f->rec32)
            return fail(FQSL_ERR_UNSUPPORTED, "%s: field not packed in the reverse sweep's precision", who);
    }
    if (p->precision != FQSL_F64 && !f->rec32)
        return fail(FQSL_ERR_UNSUPPORTED, "%s: field was not packed in FP32 (FQSL_PACK_F32)", who);
    if (p->precision == FQSL_F64 && !f->rec64)
        return fail(FQSL_ERR_UNSUPPORTED, "%s: field was not packed in FP64 (FQSL_PACK_F64)", who);
    if (p->method == 2 && p->gradb_way == 1 && !(p->precision == FQSL_F64 ? f->grad64 : f->grad32))
        return fail(FQSL_ERR_UNSUPPORTED, "%s: Method II way 1 needs a field packed with FQSL_PACK_GRADB", who);
    if (p->qperp != 0 && p->qperp != 1) return fail(FQSL_ERR_ARG, "%s: qperp must be 0 or 1", who);
    if (p->scheme != 0 && p->scheme != 1) return fail(FQSL_ERR_ARG, "%s: scheme must be 0 or 1", who);
    if (p->scheme == 1) {
        if (!(p->step > 0) || !isfinite(p->step)) return fail(FQSL_ERR_ARG, "%s: step must be > 0", who);
        if (!(p->step_min >= 0) || !(p->step_min <= p->step))
            return fail(FQSL_ERR_ARG, "%s: need 0 <= step_min <= step", who);
    }
    if (p->qperp && p->method != 2) return fail(FQSL_ERR_UNSUPPORTED, "%s: Q_perp needs Method II", who);
    if (f->g.rect && p->tape) {
        // the stretched-grid tape: the reverse sweep runs in the taped state's
        // precision (FP64 physical positions, FP32 relative ones)
        const int rp = p->reverse_precision < 0 ? p->precision : p->reverse_precision;
        if ((rp == FQSL_F64) != (p->precision == FQSL_F64))
            return fail(FQSL_ERR_UNSUPPORTED, "%s: on a stretched grid the reverse sweep runs in the taped map's "
                                              "state precision (FP64 with FP64, FP32 or FP32_ACC64 with FP32)", who);
    }
    return FQSL_OK;
}

// scheduling defaults, measured on GB300: a warp refills once all 32 lanes are
// idle (lanes that start together keep sharing cache lines; refilling single
// lanes was slower), and lanes start their second direction at once
constexpr int kDefaultRefill = 32;
constexpr int kDefaultSyncDirs = 0;

DevParams dev_params(const fqsl_params *p)
{
    DevParams d;
    d.tol = p->tol;
    d.h0 = p->h0;
    d.hmin = p->h_min;
    d.hmax = p->h_max;
    d.rot = p->rot_thresh;
    d.texp = p->tol_exp;
    d.graze = p->graze;
    d.eps2 = p->eps_way2;
    d.max_steps = p->max_steps;
    d.method = p->method;
    d.way = p->gradb_way;
    d.refill = p->refill_lanes > 0 ? p->refill_lanes : kDefaultRefill;
    d.sync_dirs = p->sync_dirs >= 0 ? p->sync_dirs : kDefaultSyncDirs;
    d.chunk = (p->chunk_tiles > 0 ? p->chunk_tiles : 1) * kTileU * kTileV;
    d.scheme = p->scheme;
    d.step = p->step;
    d.step_min = p->step_min;
    return d;
}

struct Scratch {
    LineRecs rec{}, ext{};
    SeedPrep prep{};
    int32_t *rot_seed = nullptr, *rot_slot = nullptr;
    size_t bytes = 0;
};

// Lay out the per-call scratch for n primary lines (and 4 n extra lines when
// rotation is possible): FP64 records for the FP64 tracer, index-space
// records and the seed pre-pass arrays for the FP32 tracers. With base == NULL
// only the size is computed.
Scratch layout(char *base, long long n, bool rot, bool lattice, bool f32, bool m2 = false)
{
    Carver c{base};
    Scratch s;
    LineRecs &r = s.rec;
    if (m2) {
        if (f32) {
            r.dev32 = c.take<float>(12 * n);
            s.prep.fu = c.take<float4>(n);
            s.prep.fv = c.take<float4>(n);
        } else {
            r.dev64 = c.take<double>(12 * n);
            r.be64 = c.take<double>(6 * n);
        }
    }
    if (f32) {
        r.xi1 = c.take<float>(3 * n);
        r.xi2 = c.take<float>(3 * n);
        r.kacc = c.take<float4>(2 * n);
    } else {
        r.r1 = c.take<double>(3 * n);
        r.r2 = c.take<double>(3 * n);
        r.bn1 = lattice ? c.take<double>(n) : nullptr;
        r.bn2 = lattice ? c.take<double>(n) : nullptr;
        r.tw = c.take<double>(n);
        r.len = c.take<double>(n);
    }
    r.bn0 = lattice ? c.take<double>(n) : nullptr;
    r.f1 = c.take<int8_t>(n);
    r.f2 = c.take<int8_t>(n);
    r.st = c.take<uint8_t>(n);
    r.steps = c.take<int32_t>(n);
    if (f32 && lattice) {
        s.prep.seed = c.take<float4>(n);
        s.prep.flags = c.take<uint8_t>(n);
    }
    if (rot) {
        s.rot_seed = c.take<int32_t>(n);
        s.rot_slot = c.take<int32_t>(n);
        LineRecs &x = s.ext;
        if (f32) {
            x.xi1 = c.take<float>(12 * n);
            x.xi2 = c.take<float>(12 * n);
        } else {
            x.r1 = c.take<double>(12 * n);
            x.r2 = c.take<double>(12 * n);
        }
        x.f1 = c.take<int8_t>(4 * n);
        x.f2 = c.take<int8_t>(4 * n);
        x.st = c.take<uint8_t>(4 * n);
        x.steps = c.take<int32_t>(4 * n);
    }
    s.bytes = c.off;
    return s;
}

fqsl_status ensure_scratch(fqsl_field f, size_t bytes)
{
    if (bytes <= f->scratch_cap) return FQSL_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "scratch: synchronize");
    cudaFree(f->scratch);
    f->scratch = nullptr;
    f->scratch_cap = 0;
    e = dev_malloc((void **)&f->scratch, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "scratch allocation");
    }
    f->scratch_cap = bytes;
    return FQSL_OK;
}

int blocks_per_sm(fqsl_field f, int precision, int src, int p_scheme)
{
    int &c = f->blocks_cache[p_scheme][precision][src];
    if (!c) {
        if (p_scheme == 1 && f->g.rect)
            c = precision == FQSL_F64 ? trace_rect_rk38_blocks_per_sm_f64(src)
                                      : trace_rect_rk38_blocks_per_sm_f32(src, precision == FQSL_F32_ACC64);
        else if (p_scheme == 1)
            c = precision == FQSL_F64 ? trace_rk38_blocks_per_sm_f64(src)
                                      : trace_rk38_blocks_per_sm_f32(src, precision == FQSL_F32_ACC64);
        else if (f->g.rect)
            c = precision == FQSL_F64 ? trace_rect_blocks_per_sm_f64(src)
                                      : trace_rect_blocks_per_sm_f32(src, precision == FQSL_F32_ACC64);
        else
            c = precision == FQSL_F64 ? trace_blocks_per_sm_f64(src)
                                      : trace_blocks_per_sm_f32(src, precision == FQSL_F32_ACC64);
    }
    return c;
}

cudaError_t launch_trace(fqsl_field f, const fqsl_params *p, const TraceArgs &a, int src, long long items,
                         cudaStream_t s)
{
    const long long warps_needed = (items + 31) / 32;
    int bps = blocks_per_sm(f, p->precision, src, p->scheme);
    if (p->blocks_per_sm > 0 && p->blocks_per_sm < bps) bps = p->blocks_per_sm;
    long long grid = (long long)f->sms * bps;
    const long long need = (warps_needed * 32 + kTraceBlock - 1) / kTraceBlock;
    if (src != kSrcExtra && need < grid) grid = need;
    if (grid < 1) grid = 1;
    return p->precision == FQSL_F64 ? launch_trace_f64(a, src, (int)grid, kTraceBlock, s)
                                    : launch_trace_f32(a, src, (int)grid, kTraceBlock, s,
                                                       p->precision == FQSL_F32_ACC64);
}

cudaError_t launch_trace_m2(fqsl_field f, const fqsl_params *p, const TraceArgs &a, cudaStream_t s)
{
    int &c = f->blocks_cache_m2[p->scheme][p->precision == FQSL_F64 ? 1 : 0][p->gradb_way - 1];
    if (!c) {
        if (p->scheme == 1 && f->g.rect)
            c = p->precision == FQSL_F64 ? trace_dev_rect_rk38_blocks_per_sm_f64(p->gradb_way)
                                         : trace_dev_rect_rk38_blocks_per_sm_f32(p->gradb_way);
        else if (p->scheme == 1)
            c = p->precision == FQSL_F64 ? trace_dev_rk38_blocks_per_sm_f64(p->gradb_way)
                                         : trace_dev_rk38_blocks_per_sm_f32(p->gradb_way);
        else if (f->g.rect)
            c = p->precision == FQSL_F64 ? trace_dev_rect_blocks_per_sm_f64(p->gradb_way)
                                         : trace_dev_rect_blocks_per_sm_f32(p->gradb_way);
        else
            c = p->precision == FQSL_F64 ? trace_dev_blocks_per_sm_f64(p->gradb_way)
                                         : trace_dev_blocks_per_sm_f32(p->gradb_way);
    }
    long long grid = (long long)f->sms * (p->blocks_per_sm > 0 && p->blocks_per_sm < c ? p->blocks_per_sm : c);
    const long long need = (a.nitems + kTraceBlock - 1) / kTraceBlock;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    return p->precision == FQSL_F64 ? launch_trace_dev_f64(a, p->gradb_way, (int)grid, kTraceBlock, s)
                                    : launch_trace_dev_f32(a, p->gradb_way, (int)grid, kTraceBlock, s);
}

// Does the plane x_a = x (a plane lattice's S0 normal to axis a) lie on a
// face of the box? On a uniform grid its index coordinate is 0 or n - 1; on a
// stretched grid x is the first or the last node coordinate. (The tracer
// decides rotation seed by seed; this only spares the rotated-S0 buffers and
// launch of a face plane.)
bool on_box_face(const FieldView &g, int a, double x)
{
    if (g.rect) return x == g.lo64[a] || x == g.hi64[a];
    const int na = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
    const double xi = (x - g.o[a]) / g.d[a];
    return xi == 0.0 || xi == (double)(na - 1);
}

void cross(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// The lattice in index coordinates (used by the FP32 tracer's seed set-up).
void index_lattice(const fqsl_field f, Lattice &lat)
{
    for (int a = 0; a < 3; a++) {
        lat.sdu[a] = f->g.d[a] / lat.du;
        lat.sdv[a] = f->g.d[a] / lat.dv;
        lat.sdr[a] = f->g.d[a] / lat.drot;
    }
    for (int a = 0; a < 3; a++) {
        lat.xo[a] = (lat.o[a] - f->g.o[a]) / f->g.d[a];
        lat.xa1[a] = lat.a1[a] / f->g.d[a];
        lat.xa2[a] = lat.a2[a] / f->g.d[a];
        lat.xa3[a] = lat.a3[a] / f->g.d[a];
    }
}

// Layout of a taped map in the field's tape buffer: the line records (as in
// layout()), counters, the step tape (pool chunks of k steps), the footpoint
// and extra-seed adjoints, the loss sums and the adjoint node grid. With
// rotation possible the half-lines of the 4 n extra lines follow the 2 n
// lattice half-lines.
struct TapeLayout {
    Scratch s;
    unsigned long long *ctr;  // [0] tape chunks handed out, [1] live steps of the reverse sweep,
                              // [2], [3] failed index checks of the adjoint kernels,
                              // [4] rotated seeds (as unsigned), [5] work counter of the extra tracer
    Tape tape;
    double *xbar, *xseed, *sums;
    long long halves;
    void *acc;
    size_t bytes;
};

constexpr int kDefaultTapeChunk = 16;

// The taped forward also keeps every accepted step's states and stage
// derivatives for the reverse sweep (sparing its recompute) when the reverse
// runs in the tape's precision class and the arrays, sized for the whole pool,
// stay within this budget.
constexpr size_t kKeepBudget = (size_t)4 << 30;

TapeLayout tape_layout(char *base, long long n, bool rot, bool f32, long long pool, int k, size_t nodes,
                       bool acc64, bool keep, long long wcap)
{
    TapeLayout t{};
    t.s = layout(base, n, rot, true, f32);
    Carver c{base ? base + t.s.bytes : nullptr};
    const size_t ts = f32 ? 4 : 8;
    t.halves = 2 * n + (rot ? 8 * n : 0);
    t.ctr = c.take<unsigned long long>(6);
    t.tape.k = k;
    t.tape.cap = pool;
    t.tape.next = t.ctr;
    t.tape.prev = c.take<int32_t>((size_t)pool);
    t.tape.xi = c.take<char>((size_t)pool * 4 * ts);
    t.tape.h = c.take<char>((size_t)pool * k * ts);
    t.tape.head = c.take<int4>((size_t)t.halves);
    t.tape.xe = c.take<char>((size_t)t.halves * 4 * ts);
    t.tape.owner = c.take<int32_t>((size_t)pool);
    t.tape.wx = keep ? c.take<char>((size_t)wcap * (k + 1) * kStateStride * ts) : nullptr;
    t.tape.wk = keep ? c.take<char>((size_t)wcap * k * kStageStride * ts) : nullptr;
    t.tape.wcap = keep ? wcap : 0;
    t.xbar = c.take<double>((size_t)(3 * t.halves));
    t.xseed = rot ? c.take<double>((size_t)(24 * n)) : nullptr;
    t.sums = c.take<double>(2);
    t.acc = c.take<char>(nodes * 8 * (acc64 ? 8 : 4));
    t.bytes = t.s.bytes + c.off;
    return t;
}

// the precision the reverse sweep runs in, and whether its node grid is double
int reverse_precision_of(const fqsl_params &p) { return p.reverse_precision < 0 ? p.precision : p.reverse_precision; }
bool acc64_of(const fqsl_params &p) { return reverse_precision_of(p) != FQSL_F32; }

// the taped map's layout in its tape's buffer (base NULL: sizes only)
TapeLayout tape_layout_of(const fqsl_tape t, char *base, long long pool)
{
    const fqsl_params &p = t->p;
    const long long n = t->lat.n1 * t->lat.n2 * t->lat.n3;
    const int k = p.tape_chunk > 0 ? p.tape_chunk : kDefaultTapeChunk;
    const size_t ts = p.precision == FQSL_F64 ? 8 : 4;
    const bool same = (reverse_precision_of(p) == FQSL_F64) == (p.precision == FQSL_F64);
    const size_t per_chunk = (size_t)((k + 1) * kStateStride + k * kStageStride) * ts;
    const long long wcap = t->keep_cap < 1 ? 1 : (t->keep_cap > pool ? pool : t->keep_cap);
    const bool keep = same && (size_t)wcap * per_chunk <= kKeepBudget;
    return tape_layout(base, n, t->lat.allow_rot, p.precision != FQSL_F64, pool, k, t->nodes, acc64_of(p), keep,
                       wcap);
}

fqsl_status ensure_tape_buf(fqsl_tape t, size_t bytes)
{
    if (bytes <= t->cap) return FQSL_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "tape buffer: synchronize");
    cudaFree(t->buf);
    t->buf = nullptr;
    t->cap = 0;
    e = dev_malloc((void **)&t->buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "tape buffer allocation");
    }
    t->cap = bytes;
    return FQSL_OK;
}

int tape_blocks_per_sm(fqsl_field f, int precision, int src, int p_scheme)
{
    int &c = f->blocks_cache_tape[p_scheme][precision][src == kSrcExtra ? 1 : 0];
    const bool acc64 = precision == FQSL_F32_ACC64;
    if (!c && f->g.rect && p_scheme == 1)
        c = precision == FQSL_F64 ? trace_tape_rect_rk38_blocks_per_sm_f64(src)
                                  : trace_tape_rect_rk38_blocks_per_sm_f32(src, acc64);
    else if (!c && f->g.rect)
        c = precision == FQSL_F64 ? trace_tape_rect_blocks_per_sm_f64(src) : trace_tape_rect_blocks_per_sm_f32(src, acc64);
    else if (!c && p_scheme == 1)
        c = precision == FQSL_F64 ? trace_tape_rk38_blocks_per_sm_f64(src) : trace_tape_rk38_blocks_per_sm_f32(src, acc64);
    else if (!c)
        c = precision == FQSL_F64 ? trace_tape_blocks_per_sm_f64(src) : trace_tape_blocks_per_sm_f32(src, acc64);
    return c;
}

cudaError_t launch_tape(const TraceArgs &a, const fqsl_params *p, int src, long long grid, cudaStream_t s)
{
    if (grid < 1) grid = 1;
    const bool acc64 = p->precision == FQSL_F32_ACC64;
    if (a.f.rect && p->scheme == 1)
        return p->precision == FQSL_F64 ? launch_trace_tape_rect_rk38_f64(a, src, (int)grid, s)
                                        : launch_trace_tape_rect_rk38_f32(a, src, (int)grid, s, acc64);
    if (a.f.rect)
        return p->precision == FQSL_F64 ? launch_trace_tape_rect_f64(a, src, (int)grid, s)
                                        : launch_trace_tape_rect_f32(a, src, (int)grid, s, acc64);
    if (p->scheme == 1)
        return p->precision == FQSL_F64 ? launch_trace_tape_rk38_f64(a, src, (int)grid, s)
                                        : launch_trace_tape_rk38_f32(a, src, (int)grid, s, acc64);
    return p->precision == FQSL_F64 ? launch_trace_tape_f64(a, src, (int)grid, s)
                                    : launch_trace_tape_f32(a, src, (int)grid, s, acc64);
}

// Shared body of the plane and volume Q maps (the caller holds f->mu). With a
// tape (Method I) the records live in the tape's buffer and the lattice
// tracer also writes the step tape into it.
fqsl_status run_qmap_locked(fqsl_field f, const Lattice &lat0, const fqsl_params *p, const fqsl_out *out,
                            cudaStream_t stream, bool face_plane, fqsl_tape tape, const char *who)
{
    Lattice lat = lat0;
    index_lattice(f, lat);
    const long long n = lat.n1 * lat.n2 * lat.n3;
    lat.tiles_u = (lat.n1 + kTileU - 1) / kTileU;
    lat.tiles_v = (lat.n2 + kTileV - 1) / kTileV;
    lat.allow_rot = (p->method == 1 && !face_plane) ? 1 : 0;
    const bool f32 = p->precision != FQSL_F64;
    const bool m2 = p->method == 2;
    Scratch s;
    TapeLayout tl{};
    if (tape) {
        tape->valid = false;
        tape->field = f;
        tape->field_serial = f->serial;
        tape->gen = f->gen;
        tape->lat = lat;
        tape->p = *p;
        tape->face_plane = face_plane;
        tape->nodes = (size_t)f->g.nx * f->g.ny * f->g.nz;
        const int k = p->tape_chunk > 0 ? p->tape_chunk : kDefaultTapeChunk;
        // first guess: 128 accepted steps per direction on average
        const long long guess = 2 * n * (128 / k + 1) + 1024;
        if (tape->pool < guess) tape->pool = guess;
        // the kept states: two chunks per direction at first, then what the
        // last backward call needed
        if (tape->keep_cap < 1) tape->keep_cap = 4 * n + 1024;
        if (tape->keep_want > tape->keep_cap) tape->keep_cap = tape->keep_want;
        fqsl_status st = ensure_tape_buf(tape, tape_layout_of(tape, nullptr, tape->pool).bytes);
        if (st != FQSL_OK) return st;
        tl = tape_layout_of(tape, (char *)tape->buf, tape->pool);
        s = tl.s;
    } else {
        Scratch sz = layout(nullptr, n, lat.allow_rot, true, f32, m2);
        fqsl_status st = ensure_scratch(f, sz.bytes);
        if (st != FQSL_OK) return st;
        s = layout((char *)f->scratch, n, lat.allow_rot, true, f32, m2);
    }

    cudaError_t e = cudaMemsetAsync(f->counters, 0, 4 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess && lat.allow_rot) e = cudaMemsetAsync(s.rot_slot, 0, (size_t)n * sizeof(int32_t), stream);
    if (e == cudaSuccess && tape) e = cudaMemsetAsync(tl.ctr, 0, 6 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess && tape) {
        // the taped tracer traces the two directions of a line as separate
        // items and combines status, trial count and (FP64) sums atomically
        e = cudaMemsetAsync(s.rec.st, 0, (size_t)n, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.rec.steps, 0, (size_t)n * sizeof(int32_t), stream);
        if (e == cudaSuccess && s.rec.tw) e = cudaMemsetAsync(s.rec.tw, 0, (size_t)n * sizeof(double), stream);
        if (e == cudaSuccess && s.rec.len) e = cudaMemsetAsync(s.rec.len, 0, (size_t)n * sizeof(double), stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, who);

    TraceArgs a{};
    a.f = f->g;
    a.f.rec = p->precision == FQSL_F64 ? f->rec64 : f->rec32;
    a.f.grad = p->precision == FQSL_F64 ? f->grad64 : f->grad32;
    a.p = dev_params(p);
    a.lat = lat;
    a.rec = s.rec;
    a.ext = s.ext;
    a.q.head = f->counters;
    // a taped map keeps its rotated-seed count with the tape (f->counters is
    // shared with the field's other calls)
    a.q.rot_count = tape ? (unsigned int *)(tl.ctr + 4) : (unsigned int *)(f->counters + 2);
    a.q.rot_seed = s.rot_seed;
    a.q.rot_slot = s.rot_slot;
    a.prep = s.prep;
    a.tape = tl.tape;
    a.nitems = lat.n3 * lat.tiles_u * lat.tiles_v * (long long)(kTileU * kTileV);
    if (f32) {
        e = launch_seed_prep_f32(a, n, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
    }
    mark(f, 0, stream);
    if (m2) {
        e = launch_trace_m2(f, p, a, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
        mark(f, 1, stream);
        mark(f, 2, stream);
        AssembleArgs g{};
        g.f = a.f;
        g.lat = lat;
        g.rec = s.rec;
        g.out = *out;
        g.n = n;
        g.want_q = 1;
        g.qperp = p->qperp;
        e = f32 ? launch_assemble_m2_f32(g, stream) : launch_assemble_m2_f64(g, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
        mark(f, 3, stream);
        f->timed = f->timing;
        f->extra_timed = false;
        return FQSL_OK;
    }
    if (tape) {
        int bps = tape_blocks_per_sm(f, p->precision, kSrcLattice, p->scheme);
        if (p->blocks_per_sm > 0 && p->blocks_per_sm < bps) bps = p->blocks_per_sm;
        long long grid = (long long)f->sms * bps;
        a.nitems *= 2;  // one item per direction of a line
        const long long need = (a.nitems + kTraceBlock - 1) / kTraceBlock;
        if (need < grid) grid = need;
        if (grid < 1) grid = 1;
        e = launch_tape(a, p, kSrcLattice, grid, stream);
    } else {
        e = launch_trace(f, p, a, kSrcLattice, a.nitems, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 1, stream);
    if (lat.allow_rot) {
        if (tape) {
            // the extra lines' half-lines follow the lattice's on the tape;
            // their count is read on the device (persistent grid)
            a.q.head = tl.ctr + 5;
            a.tape.hl_base = 2 * n;
            int bps = tape_blocks_per_sm(f, p->precision, kSrcExtra, p->scheme);
            if (p->blocks_per_sm > 0 && p->blocks_per_sm < bps) bps = p->blocks_per_sm;
            e = launch_tape(a, p, kSrcExtra, (long long)f->sms * bps, stream);
        } else {
            a.q.head = f->counters + 1;
            e = launch_trace(f, p, a, kSrcExtra, 4 * n, stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, who);
    }
    if (tape) {
        // the chunk count, for fqsl_backward's pool check
        if (!tape->used_host) {
            e = cudaHostAlloc((void **)&tape->used_host, sizeof(unsigned long long), cudaHostAllocDefault);
            if (e != cudaSuccess) {
                tape->used_host = nullptr;
                return cuda_fail(e, who);
            }
        }
        if (!tape->used_ev) {
            e = cudaEventCreateWithFlags(&tape->used_ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                tape->used_ev = nullptr;
                return cuda_fail(e, who);
            }
        }
        e = cudaMemcpyAsync(tape->used_host, tl.ctr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaEventRecord(tape->used_ev, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
    }
    mark(f, 2, stream);
    AssembleArgs g{};
    g.f = a.f;
    g.lat = lat;
    g.rec = s.rec;
    g.ext = s.ext;
    g.rot_slot = lat.allow_rot ? s.rot_slot : nullptr;
    g.out = *out;
    g.n = n;
    g.want_q = 1;
    e = f32 ? launch_assemble_f32(g, stream) : launch_assemble(g, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 3, stream);
    f->timed = f->timing;
    f->extra_timed = lat.allow_rot != 0;
    if (tape) tape->valid = true;
    return FQSL_OK;
}

// The tape of a call that asks for one (params->tape = 1): the caller's
// *tape_or_null, or a new tape stored there. *created tells a failing call to
// release a tape it made.
fqsl_status take_tape(const fqsl_params *p, fqsl_tape *tape_or_null, fqsl_tape *t, bool *created, const char *who)
{
    *t = nullptr;
    *created = false;
    if (!p->tape) return FQSL_OK;
    if (p->method != 1) return fail(FQSL_ERR_UNSUPPORTED, "%s: the step tape needs Method I", who);
    if (!tape_or_null) return fail(FQSL_ERR_ARG, "%s: params.tape = 1 needs a tape (tape_or_null)", who);
    if (!*tape_or_null) {
        *tape_or_null = new (std::nothrow) fqsl_tape_s();
        if (!*tape_or_null) return fail(FQSL_ERR_OOM, "%s: host allocation of the tape", who);
        *created = true;
    }
    *t = *tape_or_null;
    return FQSL_OK;
}

void release_tape(fqsl_tape t)
{
    if (!t) return;
    cudaFree(t->buf);
    cudaFree(t->work);
    if (t->used_host) cudaFreeHost(t->used_host);
    if (t->used_ev) cudaEventDestroy(t->used_ev);
    delete t;
}

fqsl_status run_qmap(fqsl_field f, const Lattice &lat0, const fqsl_params *p, const fqsl_out *out,
                     cudaStream_t stream, bool face_plane, const char *who, fqsl_tape *tape_or_null)
{
    fqsl_tape t = nullptr;
    bool created = false;
    fqsl_status st = take_tape(p, tape_or_null, &t, &created, who);
    if (st != FQSL_OK) return st;
    {
        std::lock_guard<std::mutex> lock(f->mu);
        st = run_qmap_locked(f, lat0, p, out, stream, face_plane, t, who);
    }
    if (st != FQSL_OK && created) {
        release_tape(t);
        *tape_or_null = nullptr;
    }
    return st;
}

}  // namespace

extern "C" {

fqsl_status fqsl_qmap_plane(fqsl_field f, const double origin[3], const double u[3], const double v[3],
                            long long nu, long long nv, const fqsl_params *p, const fqsl_out *out,
                            fqsl_tape *tape_or_null, void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_qmap_plane";
    fqsl_status st = check_params(f, p, who);
    if (st != FQSL_OK) return st;
    if (!out) return fail(FQSL_ERR_ARG, "%s: out is NULL", who);
    if (!finite3(origin) || !finite3(u) || !finite3(v)) return fail(FQSL_ERR_ARG, "%s: non-finite plane", who);
    if (!count_ok(nu, nv, kMaxCount)) return fail(FQSL_ERR_ARG, "%s: need nu, nv >= 1 and nu*nv < 2^31", who);
    double n0[3];
    cross(u, v, n0);
    const double nn = sqrt(n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2]);
    const double nuu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double nvv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(nuu > 0) || !(nvv > 0) || !(nn > 0)) return fail(FQSL_ERR_ARG, "%s: u and v must span a plane", who);
    if (fabs(u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) > 1e-12 * nuu * nvv)
        return fail(FQSL_ERR_ARG, "%s: u and v must be orthogonal", who);
    Lattice lat{};
    for (int a = 0; a < 3; a++) {
        lat.o[a] = origin[a];
        lat.a1[a] = u[a];
        lat.a2[a] = v[a];
        lat.a3[a] = 0.0;
        lat.n0[a] = n0[a] / nn;
    }
    lat.n1 = nu;
    lat.n2 = nv;
    lat.n3 = 1;
    lat.du = nuu;
    lat.dv = nvv;
    lat.drot = fmin(nuu, nvv);
    int zeros = 0, axis = -1;
    for (int a = 0; a < 3; a++) {
        if (lat.n0[a] == 0.0) zeros++;
        else axis = a;
    }
    lat.normal_axis = zeros == 2 ? axis : -1;
    bool face_plane = false;
    if (lat.normal_axis >= 0) {
        face_plane = on_box_face(f->g, lat.normal_axis, origin[lat.normal_axis]);
    }
    return run_qmap(f, lat, p, out, (cudaStream_t)cuda_stream, face_plane, who, tape_or_null);
}

fqsl_status fqsl_qmap_volume(fqsl_field f, const double origin[3], const double step[3], long long nx, long long ny,
                             long long nz, const fqsl_params *p, const fqsl_out *out, fqsl_tape *tape_or_null,
                             void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_qmap_volume";
    fqsl_status st = check_params(f, p, who);
    if (st != FQSL_OK) return st;
    if (!out) return fail(FQSL_ERR_ARG, "%s: out is NULL", who);
    if (!finite3(origin) || !finite3(step)) return fail(FQSL_ERR_ARG, "%s: non-finite lattice", who);
    if (!(step[0] > 0 && step[1] > 0 && step[2] > 0)) return fail(FQSL_ERR_ARG, "%s: steps must be > 0", who);
    if (!count_ok(nx, ny, kMaxCount) || !count_ok(nx * ny, nz, kMaxCount))
        return fail(FQSL_ERR_ARG, "%s: need nx, ny, nz >= 1 and nx*ny*nz < 2^31", who);
    Lattice lat{};
    for (int a = 0; a < 3; a++) {
        lat.o[a] = origin[a];
        lat.a1[a] = a == 0 ? step[0] : 0.0;
        lat.a2[a] = a == 1 ? step[1] : 0.0;
        lat.a3[a] = a == 2 ? step[2] : 0.0;
        lat.n0[a] = a == 2 ? 1.0 : 0.0;
    }
    lat.n1 = nx;
    lat.n2 = ny;
    lat.n3 = nz;
    lat.du = step[0];
    lat.dv = step[1];
    lat.drot = fmin(step[0], step[1]);
    lat.normal_axis = 2;
    return run_qmap(f, lat, p, out, (cudaStream_t)cuda_stream, false, who, tape_or_null);
}

fqsl_status fqsl_twist(fqsl_field f, const double *seeds_dev, long long n, const fqsl_params *p, const fqsl_out *out,
                       void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_twist";
    fqsl_status st = check_params(f, p, who);
    if (st != FQSL_OK) return st;
    if (p->tape) return fail(FQSL_ERR_UNSUPPORTED, "%s: the step tape is recorded for plane maps only", who);
    if (!out) return fail(FQSL_ERR_ARG, "%s: out is NULL", who);
    if (n < 0 || n > (1LL << 31) - 1) return fail(FQSL_ERR_ARG, "%s: n out of range", who);
    if (n == 0) return FQSL_OK;
    if (!seeds_dev) return fail(FQSL_ERR_ARG, "%s: seeds_dev is NULL", who);
    if (((uintptr_t)seeds_dev) % 8) return fail(FQSL_ERR_ARG, "%s: seeds_dev must be 8-byte aligned", who);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const bool f32 = p->precision != FQSL_F64;
    std::lock_guard<std::mutex> lock(f->mu);
    Scratch sz = layout(nullptr, n, false, false, f32);
    st = ensure_scratch(f, sz.bytes);
    if (st != FQSL_OK) return st;
    Scratch s = layout((char *)f->scratch, n, false, false, f32);
    cudaError_t e = cudaMemsetAsync(f->counters, 0, 4 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    TraceArgs a{};
    a.f = f->g;
    a.f.rec = p->precision == FQSL_F64 ? f->rec64 : f->rec32;
    a.p = dev_params(p);
    a.seeds = seeds_dev;
    a.nitems = n;
    a.rec = s.rec;
    a.q.head = f->counters;
    mark(f, 0, stream);
    e = launch_trace(f, p, a, kSrcList, n, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 1, stream);
    mark(f, 2, stream);
    AssembleArgs g{};
    g.f = a.f;
    g.lat.n1 = n;
    g.lat.n2 = 1;
    g.lat.n3 = 1;
    g.rec = s.rec;
    g.out = *out;
    g.out.Q = nullptr;
    g.n = n;
    g.want_q = 0;
    e = f32 ? launch_assemble_f32(g, stream) : launch_assemble(g, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 3, stream);
    f->timed = f->timing;
    f->extra_timed = false;
    return FQSL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fqsl_qmap_plane_static: the plane map with its scratch in a static device
// array, for callers that cannot allocate device memory.
// ---------------------------------------------------------------------------
namespace {

// 323 bytes per seed for 65536 seeds with rotation buffers, plus counters and
// the 256-byte alignment of each carved array
constexpr size_t kStaticScratchBytes = (size_t)22 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
char *g_static_addr[kMaxDevices] = {};

// Device address of the static array on the current device (looked up once).
fqsl_status static_scratch(char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "fqsl_qmap_plane_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(FQSL_ERR_UNSUPPORTED, "fqsl_qmap_plane_static: device %d", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "fqsl_qmap_plane_static: cudaGetSymbolAddress");
        g_static_addr[dev] = (char *)ptr;
    }
    *out = g_static_addr[dev];
    return FQSL_OK;
}

}  // namespace

extern "C" fqsl_status fqsl_qmap_plane_static(fqsl_field f, const double origin[3], const double u[3],
                                              const double v[3], long long nu, long long nv, const fqsl_params *p,
                                              const fqsl_out *out, void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_qmap_plane_static";
    fqsl_status st = check_params(f, p, who);
    if (st != FQSL_OK) return st;
    if (p->tape) return fail(FQSL_ERR_UNSUPPORTED, "%s: no step tape without allocation", who);
    if (p->method != 1) return fail(FQSL_ERR_UNSUPPORTED, "%s: Method I only", who);
    if (!out) return fail(FQSL_ERR_ARG, "%s: out is NULL", who);
    if (!finite3(origin) || !finite3(u) || !finite3(v)) return fail(FQSL_ERR_ARG, "%s: non-finite plane", who);
    if (nu < 1 || nv < 1) return fail(FQSL_ERR_ARG, "%s: need nu, nv >= 1", who);
    if (!count_ok(nu, nv, FQSL_STATIC_MAX_SEEDS))
        return fail(FQSL_ERR_ARG, "%s: nu*nv (nu = %lld, nv = %lld) exceeds FQSL_STATIC_MAX_SEEDS = %d", who, nu, nv,
                    FQSL_STATIC_MAX_SEEDS);
    double n0[3];
    cross(u, v, n0);
    const double nn = sqrt(n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2]);
    const double nuu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double nvv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(nuu > 0) || !(nvv > 0) || !(nn > 0)) return fail(FQSL_ERR_ARG, "%s: u and v must span a plane", who);
    if (fabs(u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) > 1e-12 * nuu * nvv)
        return fail(FQSL_ERR_ARG, "%s: u and v must be orthogonal", who);
    Lattice lat{};
    for (int a = 0; a < 3; a++) {
        lat.o[a] = origin[a];
        lat.a1[a] = u[a];
        lat.a2[a] = v[a];
        lat.a3[a] = 0.0;
        lat.n0[a] = n0[a] / nn;
    }
    lat.n1 = nu;
    lat.n2 = nv;
    lat.n3 = 1;
    lat.du = nuu;
    lat.dv = nvv;
    lat.drot = fmin(nuu, nvv);
    int zeros = 0, axis = -1;
    for (int a = 0; a < 3; a++) {
        if (lat.n0[a] == 0.0) zeros++;
        else axis = a;
    }
    lat.normal_axis = zeros == 2 ? axis : -1;
    bool face_plane = false;
    if (lat.normal_axis >= 0) {
        face_plane = on_box_face(f->g, lat.normal_axis, origin[lat.normal_axis]);
    }
    const long long n = nu * nv;
    index_lattice(f, lat);
    lat.tiles_u = (lat.n1 + kTileU - 1) / kTileU;
    lat.tiles_v = (lat.n2 + kTileV - 1) / kTileV;
    lat.allow_rot = (p->method == 1 && !face_plane) ? 1 : 0;

    char *base = nullptr;
    st = static_scratch(&base);
    if (st != FQSL_OK) return st;
    // counters first, then the line records
    unsigned long long *counters = (unsigned long long *)base;
    const size_t head = 256;
    const bool f32 = p->precision != FQSL_F64;
    Scratch need = layout(nullptr, n, lat.allow_rot, true, f32);
    if (head + need.bytes > kStaticScratchBytes)
        return fail(FQSL_ERR_ARG, "%s: %lld seeds need %zu scratch bytes, the static array holds %zu", who, n,
                    head + need.bytes, kStaticScratchBytes);
    Scratch s = layout(base + head, n, lat.allow_rot, true, f32);
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    std::lock_guard<std::mutex> lock(f->mu);
    cudaError_t e = cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess && lat.allow_rot) e = cudaMemsetAsync(s.rot_slot, 0, (size_t)n * sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    TraceArgs a{};
    a.f = f->g;
    a.f.rec = p->precision == FQSL_F64 ? f->rec64 : f->rec32;
    a.p = dev_params(p);
    a.lat = lat;
    a.rec = s.rec;
    a.ext = s.ext;
    a.q.head = counters;
    a.q.rot_count = (unsigned int *)(counters + 2);
    a.q.rot_seed = s.rot_seed;
    a.q.rot_slot = s.rot_slot;
    a.prep = s.prep;
    a.nitems = lat.n3 * lat.tiles_u * lat.tiles_v * (long long)(kTileU * kTileV);
    if (f32) {
        e = launch_seed_prep_f32(a, n, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
    }
    mark(f, 0, stream);
    e = launch_trace(f, p, a, kSrcLattice, a.nitems, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 1, stream);
    if (lat.allow_rot) {
        a.q.head = counters + 1;
        e = launch_trace(f, p, a, kSrcExtra, 4 * n, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
    }
    mark(f, 2, stream);
    AssembleArgs g{};
    g.f = a.f;
    g.lat = lat;
    g.rec = s.rec;
    g.ext = s.ext;
    g.rot_slot = lat.allow_rot ? s.rot_slot : nullptr;
    g.out = *out;
    g.n = n;
    g.want_q = 1;
    e = f32 ? launch_assemble_f32(g, stream) : launch_assemble(g, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 3, stream);
    f->timed = f->timing;
    f->extra_timed = lat.allow_rot != 0;
    return FQSL_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct fqsl_batch_s {
    int nent = 0;
    int sms = 0;
    fqsl_params params{};
    long long total_seeds = 0, total_items = 0;
    bool any_rot = false;
    void *mem = nullptr;  // scratch of all entries, descriptors and prefixes
    TraceArgs *d_desc = nullptr;
    AssembleArgs *d_adesc = nullptr;
    long long *d_ibase = nullptr, *d_nbase = nullptr, *d_xbase = nullptr;
    unsigned long long *d_heads = nullptr;
    unsigned *d_rot_counts = nullptr;
    int32_t *d_rot_slots = nullptr;
    size_t rot_slot_bytes = 0;
    int grid = 0;
};

namespace {

// Lattice of one plane entry (the checks of fqsl_qmap_plane).
fqsl_status plane_lattice(const fqsl_field f, const fqsl_plane &pl, const fqsl_params *p, Lattice &lat,
                          const char *who)
{
    const double *origin = pl.origin, *u = pl.u, *v = pl.v;
    const long long nu = pl.nu, nv = pl.nv;
    if (!finite3(origin) || !finite3(u) || !finite3(v)) return fail(FQSL_ERR_ARG, "%s: non-finite plane", who);
    if (!count_ok(nu, nv, kMaxCount)) return fail(FQSL_ERR_ARG, "%s: need nu, nv >= 1 and nu*nv < 2^31", who);
    double n0[3];
    cross(u, v, n0);
    const double nn = sqrt(n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2]);
    const double nuu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double nvv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(nuu > 0) || !(nvv > 0) || !(nn > 0)) return fail(FQSL_ERR_ARG, "%s: u and v must span a plane", who);
    if (fabs(u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) > 1e-12 * nuu * nvv)
        return fail(FQSL_ERR_ARG, "%s: u and v must be orthogonal", who);
    lat = Lattice{};
    for (int a = 0; a < 3; a++) {
        lat.o[a] = origin[a];
        lat.a1[a] = u[a];
        lat.a2[a] = v[a];
        lat.a3[a] = 0.0;
        lat.n0[a] = n0[a] / nn;
    }
    lat.n1 = nu;
    lat.n2 = nv;
    lat.n3 = 1;
    lat.du = nuu;
    lat.dv = nvv;
    lat.drot = fmin(nuu, nvv);
    int zeros = 0, axis = -1;
    for (int a = 0; a < 3; a++) {
        if (lat.n0[a] == 0.0) zeros++;
        else axis = a;
    }
    lat.normal_axis = zeros == 2 ? axis : -1;
    bool face_plane = false;
    if (lat.normal_axis >= 0) {
        face_plane = on_box_face(f->g, lat.normal_axis, origin[lat.normal_axis]);
    }
    index_lattice(f, lat);
    lat.tiles_u = (lat.n1 + kTileU - 1) / kTileU;
    lat.tiles_v = (lat.n2 + kTileV - 1) / kTileV;
    lat.allow_rot = (p->method == 1 && !face_plane) ? 1 : 0;
    return FQSL_OK;
}

void batch_free(fqsl_batch b)
{
    if (!b) return;
    cudaFree(b->mem);
    delete b;
}

}  // namespace

extern "C" fqsl_status fqsl_batch_create(const fqsl_field *fields, const fqsl_plane *planes, const fqsl_out *outs,
                                         int n, const fqsl_params *p, fqsl_batch *out)
{
    g_err.clear();
    const char *who = "fqsl_batch_create";
    if (!out) return fail(FQSL_ERR_ARG, "%s: out is NULL", who);
    *out = nullptr;
    if (!fields || !planes || !outs || n < 1) return fail(FQSL_ERR_ARG, "%s: need n >= 1 fields, planes, outs", who);
    if (!p) return fail(FQSL_ERR_ARG, "%s: NULL params", who);
    if (p->method != 1) return fail(FQSL_ERR_UNSUPPORTED, "%s: batches run Method I", who);
    const bool f32 = p->precision != FQSL_F64;
    std::vector<Lattice> lats(n);
    std::vector<size_t> off(n);
    size_t bytes = 0;
    fqsl_batch b = new (std::nothrow) fqsl_batch_s();
    if (!b) return fail(FQSL_ERR_OOM, "%s: host allocation", who);
    b->nent = n;
    b->params = *p;
    std::vector<long long> ibase(n + 1), nbase(n + 1);
    if (p->tape) {
        delete b;
        return fail(FQSL_ERR_UNSUPPORTED, "%s: batches record no step tape", who);
    }
    for (int k = 0; k < n; k++) {
        fqsl_status st = check_params(fields[k], p, who);
        if (st != FQSL_OK) {
            delete b;
            return st;
        }
        if (fields[k]->g.rect) {
            delete b;
            return fail(FQSL_ERR_UNSUPPORTED, "%s: batches take uniform grids only", who);
        }
        st = plane_lattice(fields[k], planes[k], p, lats[k], who);
        if (st != FQSL_OK) {
            delete b;
            return st;
        }
        const long long nk = lats[k].n1 * lats[k].n2;
        ibase[k] = b->total_items;
        nbase[k] = b->total_seeds;
        b->total_items += lats[k].tiles_u * lats[k].tiles_v * (long long)(kTileU * kTileV);
        b->total_seeds += nk;
        off[k] = bytes;
        bytes += layout(nullptr, nk, lats[k].allow_rot, true, f32).bytes;
        if (lats[k].allow_rot) b->any_rot = true;
    }
    ibase[n] = b->total_items;
    nbase[n] = b->total_seeds;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    // one allocation: entry scratch, contiguous rot_slot arrays, descriptors, prefixes, counters
    const size_t rot_off = align_up(bytes);
    b->rot_slot_bytes = b->any_rot ? align_up((size_t)b->total_seeds * sizeof(int32_t)) : 0;
    const size_t desc_off = align_up(rot_off + b->rot_slot_bytes);
    const size_t adesc_off = align_up(desc_off + n * sizeof(TraceArgs));
    const size_t ib_off = align_up(adesc_off + n * sizeof(AssembleArgs));
    const size_t nb_off = align_up(ib_off + (n + 1) * sizeof(long long));
    const size_t xb_off = align_up(nb_off + (n + 1) * sizeof(long long));
    const size_t rc_off = align_up(xb_off + (n + 1) * sizeof(long long));
    const size_t hd_off = align_up(rc_off + n * sizeof(unsigned));
    const size_t total = align_up(hd_off + 4 * sizeof(unsigned long long));
    cudaError_t e = dev_malloc((void **)&b->mem, total);
    if (e != cudaSuccess) {
        delete b;
        cudaGetLastError();
        return cuda_fail(e, who);
    }
    char *base = (char *)b->mem;
    b->d_rot_slots = b->any_rot ? (int32_t *)(base + rot_off) : nullptr;
    b->d_desc = (TraceArgs *)(base + desc_off);
    b->d_adesc = (AssembleArgs *)(base + adesc_off);
    b->d_ibase = (long long *)(base + ib_off);
    b->d_nbase = (long long *)(base + nb_off);
    b->d_xbase = (long long *)(base + xb_off);
    b->d_rot_counts = (unsigned *)(base + rc_off);
    b->d_heads = (unsigned long long *)(base + hd_off);
    std::vector<TraceArgs> desc(n);
    std::vector<AssembleArgs> adesc(n);
    for (int k = 0; k < n; k++) {
        const fqsl_field f = fields[k];
        const long long nk = lats[k].n1 * lats[k].n2;
        Scratch s = layout(base + off[k], nk, lats[k].allow_rot, true, f32);
        if (lats[k].allow_rot) s.rot_slot = b->d_rot_slots + nbase[k];
        TraceArgs &a = desc[k];
        a = TraceArgs{};
        a.f = f->g;
        a.f.rec = p->precision == FQSL_F64 ? f->rec64 : f->rec32;
        a.p = dev_params(p);
        a.lat = lats[k];
        a.rec = s.rec;
        a.ext = s.ext;
        a.q.rot_count = b->d_rot_counts + k;
        a.q.rot_seed = s.rot_seed;
        a.q.rot_slot = s.rot_slot;
        a.prep = s.prep;
        a.nitems = ibase[k + 1] - ibase[k];
        AssembleArgs &g = adesc[k];
        g = AssembleArgs{};
        g.f = a.f;
        g.lat = lats[k];
        g.rec = s.rec;
        g.ext = s.ext;
        g.rot_slot = lats[k].allow_rot ? s.rot_slot : nullptr;
        g.out = outs[k];
        g.n = nk;
        g.want_q = 1;
    }
    e = cudaMemcpy(b->d_desc, desc.data(), n * sizeof(TraceArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_adesc, adesc.data(), n * sizeof(AssembleArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ibase, ibase.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_nbase, nbase.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, who);
    }
    const int bps = p->precision == FQSL_F64 ? batch_trace_blocks_per_sm_f64(p->scheme)
                                             : batch_trace_blocks_per_sm_f32(p->precision == FQSL_F32_ACC64, p->scheme);
    b->grid = b->sms * (p->blocks_per_sm > 0 && p->blocks_per_sm < bps ? p->blocks_per_sm : bps);
    *out = b;
    return FQSL_OK;
}

extern "C" fqsl_status fqsl_batch_run(fqsl_batch b, void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_batch_run";
    if (!b) return fail(FQSL_ERR_ARG, "%s: NULL batch", who);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const fqsl_params *p = &b->params;
    const bool f32 = p->precision != FQSL_F64;
    cudaError_t e = cudaMemsetAsync(b->d_heads, 0, 4 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_rot_counts, 0, b->nent * sizeof(unsigned), s);
    if (e == cudaSuccess && b->any_rot) e = cudaMemsetAsync(b->d_rot_slots, 0, b->rot_slot_bytes, s);
    if (e == cudaSuccess && f32) e = launch_batch_seed_prep_f32(b->d_desc, b->d_nbase, b->nent, b->total_seeds, s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    TraceArgs a0{};
    a0.p = dev_params(p);
    a0.p.chunk = kTileU * kTileV;  // a grab never spans two entries
    a0.q.head = b->d_heads;
    a0.nitems = b->total_items;
    BatchArgs ba{b->d_desc, b->d_ibase, b->nent};
    long long grid = b->grid;
    const long long need = (b->total_items + kTraceBlock - 1) / kTraceBlock;
    if (need < grid) grid = need;
    e = f32 ? launch_batch_trace_f32(a0, ba, kSrcLattice, p->precision == FQSL_F32_ACC64, (int)grid, s)
            : launch_batch_trace_f64(a0, ba, kSrcLattice, (int)grid, s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (b->any_rot) {
        e = launch_batch_extra_prefix(b->d_rot_counts, b->nent, b->d_xbase, s);
        if (e != cudaSuccess) return cuda_fail(e, who);
        a0.q.head = b->d_heads + 1;
        BatchArgs bx{b->d_desc, b->d_xbase, b->nent};
        e = f32 ? launch_batch_trace_f32(a0, bx, kSrcExtra, p->precision == FQSL_F32_ACC64, b->grid, s)
                : launch_batch_trace_f64(a0, bx, kSrcExtra, b->grid, s);
        if (e != cudaSuccess) return cuda_fail(e, who);
    }
    e = f32 ? launch_batch_assemble_f32(b->d_adesc, b->d_nbase, b->nent, b->total_seeds, s)
            : launch_batch_assemble_f64(b->d_adesc, b->d_nbase, b->nent, b->total_seeds, s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return FQSL_OK;
}

extern "C" fqsl_status fqsl_batch_destroy(fqsl_batch b)
{
    g_err.clear();
    if (!b) return fail(FQSL_ERR_ARG, "fqsl_batch_destroy: NULL batch");
    cudaDeviceSynchronize();
    batch_free(b);
    return FQSL_OK;
}

// ---------------------------------------------------------------------------
// fqsl_backward: reverse mode of a taped plane or volume map
// ---------------------------------------------------------------------------
extern "C" fqsl_status fqsl_backward(fqsl_field f, fqsl_tape tp, const double *dQ_dev, const double *dTw_dev,
                                     void *dB_dev, fqsl_dtype db_dtype, void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_backward";
    if (!f) return fail(FQSL_ERR_ARG, "%s: NULL field", who);
    if (!tp) return fail(FQSL_ERR_ARG, "%s: NULL tape", who);
    if (!dB_dev) return fail(FQSL_ERR_ARG, "%s: dB_dev is NULL", who);
    if (db_dtype != FQSL_F32 && db_dtype != FQSL_F64)
        return fail(FQSL_ERR_ARG, "%s: db_dtype must be FQSL_F32 or FQSL_F64", who);
    if (((uintptr_t)dB_dev) % 16) return fail(FQSL_ERR_ARG, "%s: dB_dev must be 16-byte aligned", who);
    if ((dQ_dev && ((uintptr_t)dQ_dev) % 8) || (dTw_dev && ((uintptr_t)dTw_dev) % 8))
        return fail(FQSL_ERR_ARG, "%s: dQ_dev and dTw_dev must be 8-byte aligned", who);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lock(f->mu);
    if (!tp->valid) return fail(FQSL_ERR_ARG, "%s: the tape holds no complete taped map", who);
    if (tp->field != f || tp->field_serial != f->serial)
        return fail(FQSL_ERR_ARG, "%s: the tape was recorded on another field", who);
    if (tp->gen != f->gen)
        return fail(FQSL_ERR_ARG, "%s: the field was updated after the taped map (trace it again)", who);
    const fqsl_params p = tp->p;
    const size_t nodes = (size_t)f->g.nx * f->g.ny * f->g.nz;
    const int rp = reverse_precision_of(p);
    const bool acc64 = acc64_of(p);
    const int mode = rp == FQSL_F64 ? 2 : (acc64 ? 1 : 0);
    const bool tape_f64 = p.precision == FQSL_F64;
    // The pool of the taped call must have held every chunk; if not, trace the
    // same map again with a larger pool (the map is deterministic). The clears
    // of the adjoint buffers and the Q-assembly VJP do not depend on the chunk
    // count, so they are queued before the host waits for the taped call's
    // tracers: the GPU has them to run while the host wakes and launches the
    // reverse sweep.
    unsigned long long used = 0;
    TapeLayout tl{};
    AdjArgs a{};
    for (int attempt = 0;; attempt++) {
        if (!tp->used_ev || !tp->used_host) return fail(FQSL_ERR_ARG, "%s: the tape holds no complete taped map", who);
        tl = tape_layout_of(tp, (char *)tp->buf, tp->pool);
        const Lattice &lat = tp->lat;
        const long long n = lat.n1 * lat.n2 * lat.n3;
        cudaError_t e = cudaMemsetAsync(tl.xbar, 0, (size_t)(3 * tl.halves) * sizeof(double), stream);
        if (e == cudaSuccess && tl.xseed) e = cudaMemsetAsync(tl.xseed, 0, (size_t)(24 * n) * sizeof(double), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(tl.acc, 0, nodes * 8 * (acc64 ? 8 : 4), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(tl.ctr + 1, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
        a = AdjArgs{};
        a.f = f->g;
        a.f.rec = rp == FQSL_F64 ? f->rec64 : f->rec32;
        a.f.grad = nullptr;
        a.f.err = f->counters + 4;  // the field's record of failed index checks (fqsl_field_check)
        a.p = dev_params(&p);
        a.lat = lat;
        a.rec = tl.s.rec;
        a.prep = tl.s.prep;
        a.tape = tl.tape;
        a.dQ = dQ_dev;
        a.dTw = dTw_dev;
        a.xbar = tl.xbar;
        a.acc = tl.acc;
        a.n = n;
        if (lat.allow_rot) {
            a.ext = tl.s.ext;
            a.rot_slot = tl.s.rot_slot;
            a.rot_seed = tl.s.rot_seed;
            a.rot_count = (const unsigned *)(tl.ctr + 4);
            a.xseed = tl.xseed;
        }
        e = launch_q_vjp(a, mode, tape_f64, stream);
        if (e != cudaSuccess) return cuda_fail(e, who);
        // the taped call copied its chunk count once its tracers finished
        e = cudaEventSynchronize(tp->used_ev);
        if (e != cudaSuccess) return cuda_fail(e, who);
        used = *(volatile unsigned long long *)tp->used_host;
        if (used <= (unsigned long long)tp->pool) break;
        if (attempt >= 2) return fail(FQSL_ERR_CUDA, "%s: step tape pool still exhausted after re-tracing", who);
        tp->pool = (long long)(used + used / 4 + 1024);
        const Lattice lat0 = tp->lat;
        const fqsl_out none{};
        fqsl_status st = run_qmap_locked(f, lat0, &p, &none, stream, tp->face_plane, tp, who);
        if (st != FQSL_OK) return st;
    }
    // per-step work arrays of the reverse sweep for the chunks in use (the
    // states and stage derivatives are the tape's own when the forward kept them)
    const int K = tl.tape.k;
    const size_t rs = rp == FQSL_F64 ? 8 : 4;
    const bool stored = tl.tape.wx != nullptr && (long long)used <= tl.tape.wcap;
    // the next taped call keeps as many chunks as this map used, with room
    const long long want = (long long)(used + used / 4 + 1024);
    if (want > tp->keep_want) tp->keep_want = want;
    const size_t bx = stored ? 0 : align_up((size_t)used * (K + 1) * kStateStride * rs),
                 bj = align_up((size_t)used * K * 12 * rs),
                 bk = stored ? 0 : align_up((size_t)used * K * kStageStride * rs), bb = align_up((size_t)used * K * 3 * rs),
                 bi = align_up((size_t)used * sizeof(int4)), bs = align_up((size_t)used * K * sizeof(int32_t));
    const size_t wbytes = bx + bj + bk + bb + bi + bs;
    if (wbytes > tp->work_cap) {
        cudaError_t e0 = cudaDeviceSynchronize();
        if (e0 == cudaSuccess) {
            cudaFree(tp->work);
            tp->work = nullptr;
            tp->work_cap = 0;
            e0 = dev_malloc((void **)&tp->work, wbytes);
        }
        if (e0 != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e0, "fqsl_backward: work arrays");
        }
        tp->work_cap = wbytes;
    }
    a.chunks = (long long)used;
    a.stored = stored ? 1 : 0;
    a.wx = stored ? tl.tape.wx : tp->work;
    a.wj = (char *)tp->work + bx;
    a.wk = stored ? tl.tape.wk : (char *)tp->work + bx + bj;
    a.wb = (char *)tp->work + bx + bj + bk;
    a.cinfo = (int4 *)((char *)tp->work + bx + bj + bk + bb);
    a.steps = (int32_t *)((char *)tp->work + bx + bj + bk + bb + bi);
    a.nsteps = tl.ctr + 1;  // cleared above
    cudaError_t e = cudaSuccess;
    mark(f, 0, stream);
    e = launch_reverse(a, mode, tape_f64, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 1, stream);
    mark(f, 2, stream);
    e = launch_curl_adjoint(tl.acc, acc64, f->g, dB_dev, db_dtype, stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    mark(f, 3, stream);
    f->timed = f->timing;
    f->extra_timed = false;
    return FQSL_OK;
}

extern "C" fqsl_status fqsl_tape_export(fqsl_tape tp, int cap, int32_t *nsteps_dev, int32_t *code_dev,
                                        double *hx_dev, double *h_dev, void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_tape_export";
    if (!tp) return fail(FQSL_ERR_ARG, "%s: NULL tape", who);
    if (cap < 0) return fail(FQSL_ERR_ARG, "%s: cap < 0", who);
    if (!nsteps_dev || !code_dev || !hx_dev || (cap > 0 && !h_dev))
        return fail(FQSL_ERR_ARG, "%s: NULL output", who);
    if (!tp->valid) return fail(FQSL_ERR_ARG, "%s: the tape holds no complete taped map", who);
    TapeLayout tl = tape_layout_of(tp, (char *)tp->buf, tp->pool);
    const long long n = tp->lat.n1 * tp->lat.n2 * tp->lat.n3;
    cudaError_t e = launch_tape_export(tl.tape, tp->p.precision == FQSL_F64, tl.s.rec.st, 2 * n, cap, nsteps_dev,
                                       code_dev, hx_dev, h_dev, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return FQSL_OK;
}

extern "C" fqsl_status fqsl_tape_destroy(fqsl_tape tp)
{
    g_err.clear();
    if (!tp) return fail(FQSL_ERR_ARG, "fqsl_tape_destroy: NULL tape");
    cudaDeviceSynchronize();
    release_tape(tp);
    return FQSL_OK;
}

extern "C" fqsl_status fqsl_loss_logq_tw(long long n, const double *Q_dev, const double *Tw_dev,
                                         const double *Qt_dev, const double *Twt_dev, const uint8_t *status_dev,
                                         double w_tw, double *sums_dev, double *loss_dev, double *dQ_dev,
                                         double *dTw_dev, void *cuda_stream)
{
    g_err.clear();
    const char *who = "fqsl_loss_logq_tw";
    if (n < 0) return fail(FQSL_ERR_ARG, "%s: n < 0", who);
    if (!Q_dev || !Tw_dev || !Qt_dev || !Twt_dev || !sums_dev)
        return fail(FQSL_ERR_ARG, "%s: Q, Tw, Q_target, Tw_target and sums are required", who);
    if (!isfinite(w_tw)) return fail(FQSL_ERR_ARG, "%s: w_tw must be finite", who);
    cudaError_t e = launch_loss(n, Q_dev, Tw_dev, Qt_dev, Twt_dev, status_dev, w_tw, sums_dev, loss_dev, dQ_dev,
                                dTw_dev, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return FQSL_OK;
}

extern "C" fqsl_status fqsl_field_check(fqsl_field f, void *cuda_stream)
{
    g_err.clear();
    if (!f) return fail(FQSL_ERR_ARG, "fqsl_field_check: NULL handle");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "fqsl_field_check");
    std::lock_guard<std::mutex> lock(f->mu);
    // index checks of the adjoint kernels (cleared here)
    unsigned long long w[2] = {0, 0};
    e = cudaMemcpy(w, f->counters + 4, sizeof w, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && w[1]) e = cudaMemset(f->counters + 4, 0, sizeof w);
    if (e != cudaSuccess) return cuda_fail(e, "fqsl_field_check");
    if (w[1])
        return fail(FQSL_ERR_CUDA, "fqsl_field_check: %llu failed index checks in the adjoint kernels, first: "
                                   "check %llu, value %lld", w[1], w[0] >> 56, (long long)(w[0] & ((1ull << 56) - 1)));
    return FQSL_OK;
}
