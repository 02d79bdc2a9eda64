// sn_setup.cu -- problem set-up of the C ABI: validation, level-symmetric quadrature,
// hyperplane tables, device buffers; errors and handle lifetime.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sn_internal.cuh"

namespace sn {

static thread_local std::string g_last_error;

void set_global_error(const std::string &msg) { g_last_error = msg; }

sn_status fail(sn_handle h, sn_status s, const std::string &msg)
{
    if (h) h->err = msg;
    g_last_error = msg;
    return s;
}

sn_status cuda_fail(sn_handle h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? SN_ENOMEM : SN_ECUDA, m);
}

// ---------------------------------------------------------------------------------
// Level-symmetric LQ_N set (the paper leaves the S_N set open, Sec. 2 after (9)).
// One octant holds the points (mu_i, mu_j, mu_k), i + j + k = N/2 + 2, with
// mu_i^2 = mu_1^2 + (i - 1) * 2 (1 - 3 mu_1^2) / (N - 2) and the standard mu_1.
// Points that are permutations of one another form a weight class; the class
// weights make sum w mu_x^(2m) = 1/(2m+1) hold for m = 0 and m = 2..K (K classes).
// Ordering: octant-major (bit 0: mu<0, bit 1: eta<0, bit 2: xi<0), i then j ascending.
// ---------------------------------------------------------------------------------
static bool solve_dense(int n, std::vector<long double> a, std::vector<long double> r,
                        std::vector<long double> &x)
{
    // row-reduction with partial pivoting in long double
    for (int c = 0; c < n; ++c) {
        int best = c;
        for (int i = c + 1; i < n; ++i)
            if (fabsl(a[i * n + c]) > fabsl(a[best * n + c])) best = i;
        if (a[best * n + c] == 0.0L) return false;
        for (int j = 0; j < n; ++j) std::swap(a[c * n + j], a[best * n + j]);
        std::swap(r[c], r[best]);
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            long double f = a[i * n + c] / a[c * n + c];
            for (int j = c; j < n; ++j) a[i * n + j] -= f * a[c * n + j];
            r[i] -= f * r[c];
        }
    }
    x.resize(n);
    for (int i = 0; i < n; ++i) x[i] = r[i] / a[i * n + i];
    return true;
}

static bool level_symmetric(int N, std::vector<double> &om, std::vector<double> &w)
{
    double mu1;
    switch (N) {
    case 2: mu1 = 1.0 / std::sqrt(3.0); break;
    case 4: mu1 = 0.3500212; break;
    case 6: mu1 = 0.2666355; break;
    case 8: mu1 = 0.2182179; break;
    case 10: mu1 = 0.1893213; break;
    case 12: mu1 = 0.1672126; break;
    default: return false;
    }
    const int half = N / 2;
    std::vector<long double> musq(half);
    for (int i = 0; i < half; ++i)
        musq[i] = (long double)mu1 * mu1 + (N > 2 ? i * 2.0L * (1.0L - 3.0L * mu1 * mu1) / (N - 2) : 0.0L);
    struct Pt { int l[3]; int cls; };
    std::vector<Pt> pts;
    std::vector<std::vector<int>> classes;
    for (int i = 1; i <= half; ++i)
        for (int j = 1; j <= half + 1 - i; ++j) {
            Pt p;
            p.l[0] = i; p.l[1] = j; p.l[2] = half + 2 - i - j;
            std::vector<int> key = {p.l[0], p.l[1], p.l[2]};
            std::sort(key.begin(), key.end());
            p.cls = -1;
            for (size_t c = 0; c < classes.size(); ++c)
                if (classes[c] == key) p.cls = (int)c;
            if (p.cls < 0) { p.cls = (int)classes.size(); classes.push_back(key); }
            pts.push_back(p);
        }
    const int K = (int)classes.size();
    std::vector<long double> a(K * K, 0.0L), r(K), x;
    for (int row = 0; row < K; ++row) {
        const int m = row == 0 ? 0 : row + 1;
        for (const Pt &p : pts) a[row * K + p.cls] += powl(musq[p.l[0] - 1], m);
        r[row] = 1.0L / (2 * m + 1);
    }
    if (!solve_dense(K, a, r, x)) return false;
    const int n8 = (int)pts.size();
    om.assign(8 * n8 * 3, 0.0);
    w.assign(8 * n8, 0.0);
    for (int o = 0; o < 8; ++o)
        for (int p = 0; p < n8; ++p) {
            const int d = o * n8 + p;
            for (int ax = 0; ax < 3; ++ax) {
                const double s = (o >> ax) & 1 ? -1.0 : 1.0;
                om[3 * d + ax] = s * (double)sqrtl(musq[pts[p].l[ax] - 1]);
            }
            w[d] = (double)(x[pts[p].cls] * (long double)(kPi / 2.0));
        }
    return true;
}

static bool finite_all(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

static sn_status dalloc_bytes(sn_handle h, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
    h->device_bytes += (int64_t)bytes;
    return SN_OK;
}

// n elements of the handle's element type
static sn_status dalloc(sn_handle h, void **p, size_t n) { return dalloc_bytes(h, p, n * h->esz); }

// host FP64 -> device element type
static sn_status upload(sn_handle h, void *dst, const double *src, size_t n)
{
    if (h->fp64) {
        SN_CK(h, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        return SN_OK;
    }
    std::vector<float> tmp(n);
    for (size_t i = 0; i < n; ++i) tmp[i] = (float)src[i];
    SN_CK(h, cudaMemcpyAsync(dst, tmp.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    return SN_OK;
}

template <typename T>
static sn_status upload_dirs(sn_handle h)
{
    std::vector<DirData<T>> dd(h->Do);
    for (int d = 0; d < h->Do; ++d) {
        dd[d].t3x = (T)(3.0 * std::fabs(h->omega[3 * d + 0]) / h->dx);
        dd[d].t3y = (T)(3.0 * std::fabs(h->omega[3 * d + 1]) / h->dy);
        dd[d].t3z = (T)(3.0 * std::fabs(h->omega[3 * d + 2]) / h->dz);
        dd[d].w = (T)h->w[d];
    }
    sn_status s = dalloc_bytes(h, &h->dir, sizeof(DirData<T>) * h->Do);
    if (s != SN_OK) return s;
    SN_CK(h, cudaMemcpyAsync(h->dir, dd.data(), sizeof(DirData<T>) * h->Do, cudaMemcpyHostToDevice, h->stream));
    return SN_OK;
}

static void release(sn_handle h)
{
    if (!h) return;
    for (int i = 0; i < 2; ++i)
        if (h->graphs.exec[i]) cudaGraphExecDestroy(h->graphs.exec[i]);
    free_adjoint(h);
    free_wave(h);
    void *bufs[] = {h->sigt, h->sigs, h->q, h->xfer, h->psi_inc, h->dir, h->dir_abs, h->plane_cells, h->plane_pos,
                    h->face, h->phi_oct, h->S, h->S_b, h->phi_b, h->acc, h->sigs_n, h->yhat, h->geom, h->vnode, h->omabs, h->geomB};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (h->acc_host) cudaFreeHost(h->acc_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int i = 0; i < 2; ++i)
        if (h->ev_sweep[i]) cudaEventDestroy(h->ev_sweep[i]);
    free_net(h);
    free_octnet(h);
}

// The sweep order of Sec. 2 in the canonical octant: cell (i',j',k') is solved on
// hyperplane s = i'+j'+k', after its three upwind neighbours on hyperplane s - 1.
void hyperplane_tables(int nx, int ny, int nz, std::vector<int64_t> &off, std::vector<uint32_t> &cells,
                       std::vector<uint32_t> &pos)
{
    const int np = nx + ny + nz - 2;
    const int64_t C = (int64_t)nx * ny * nz;
    off.assign(np + 1, 0);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) off[i + j + k + 1]++;
    for (int s = 0; s < np; ++s) off[s + 1] += off[s];
    cells.assign(C, 0u);
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                cells[fill[i + j + k]++] = (uint32_t)i | ((uint32_t)j << 10) | ((uint32_t)k << 20);
    pos.assign(C, 0u);
    for (int s = 0; s < np; ++s)
        for (int64_t q = off[s]; q < off[s + 1]; ++q) {
            const uint32_t pk = cells[q];
            const int64_t lin = (pk & 1023) + (int64_t)nx * (((pk >> 10) & 1023) + (int64_t)ny * (pk >> 20));
            pos[lin] = (uint32_t)(q - off[s]);
        }
}

}  // namespace sn

using namespace sn;

extern "C" {

const char *sn_status_string(sn_status s)
{
    switch (s) {
    case SN_OK: return "ok";
    case SN_EINVAL: return "invalid argument";
    case SN_ENOMEM: return "out of device memory";
    case SN_ECUDA: return "CUDA error";
    case SN_ENOCONV: return "not converged";
    case SN_ETIMEOUT: return "device wait timed out";
    case SN_ENAN: return "non-finite flux";
    case SN_ESTATE: return "invalid state";
    }
    return "unknown status";
}

const char *sn_last_error(sn_handle h)
{
    if (h) return h->err.c_str();
    return g_last_error.c_str();
}

sn_status sn_setup(sn_handle *out, const sn_mesh *mesh, const sn_quadrature *quad, const sn_xs *xs,
                   const sn_options *opts, void *stream)
{
    if (!out) return fail(nullptr, SN_EINVAL, "sn_setup: out is NULL");
    *out = nullptr;
    if (!mesh || !quad || !xs) return fail(nullptr, SN_EINVAL, "sn_setup: NULL argument");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || mesh->nx > 1023 || mesh->ny > 1023 ||
        mesh->nz > 1023)
        return fail(nullptr, SN_EINVAL, "sn_setup: cells per axis must be in 1..1023");
    if (!(mesh->lx > 0) || !(mesh->ly > 0) || !(mesh->lz > 0) || !std::isfinite(mesh->lx) ||
        !std::isfinite(mesh->ly) || !std::isfinite(mesh->lz))
        return fail(nullptr, SN_EINVAL, "sn_setup: box lengths must be finite and > 0");
    if (xs->ngroups < 1 || xs->ngroups > 1024)
        return fail(nullptr, SN_EINVAL, "sn_setup: ngroups must be in 1..1024");
    if (!xs->sigt || !xs->sigs || !xs->q || !xs->xfer)
        return fail(nullptr, SN_EINVAL, "sn_setup: NULL cross-section array");

    sn_handle h = new (std::nothrow) sn_handle_s();
    if (!h) return fail(nullptr, SN_ENOMEM, "sn_setup: host allocation failed");
    h->stream = (cudaStream_t)stream;
    h->fp64 = opts && opts->fp64;
    h->esz = h->fp64 ? sizeof(double) : sizeof(float);
    h->nx = mesh->nx; h->ny = mesh->ny; h->nz = mesh->nz;
    h->lx = mesh->lx; h->ly = mesh->ly; h->lz = mesh->lz;
    h->dx = h->lx / h->nx; h->dy = h->ly / h->ny; h->dz = h->lz / h->nz;
    h->ncell = (int64_t)h->nx * h->ny * h->nz;
    h->G = xs->ngroups;
    const int64_t C = h->ncell, G = h->G;

    // quadrature
    if (quad->order != 0) {
        if (!level_symmetric(quad->order, h->omega, h->w)) {
            delete h;
            return fail(nullptr, SN_EINVAL, "sn_setup: unsupported LQ_N order (2..12, even)");
        }
    } else {
        if (quad->ndir < 8 || quad->ndir % 8 || !quad->omega || !quad->w) {
            delete h;
            return fail(nullptr, SN_EINVAL, "sn_setup: explicit quadrature needs 8*n directions");
        }
        h->omega.assign(quad->omega, quad->omega + 3 * quad->ndir);
        h->w.assign(quad->w, quad->w + quad->ndir);
        const int n8 = quad->ndir / 8;
        bool ok = finite_all(quad->omega, 3 * quad->ndir) && finite_all(quad->w, quad->ndir);
        for (int o = 0; o < 8 && ok; ++o)
            for (int p = 0; p < n8 && ok; ++p)
                for (int ax = 0; ax < 3; ++ax) {
                    const double base = h->omega[3 * p + ax];
                    const double s = (o >> ax) & 1 ? -1.0 : 1.0;
                    if (!(base > 0) || h->omega[3 * (o * n8 + p) + ax] != s * base) ok = false;
                }
        for (int p = 0; p < n8 && ok; ++p)
            for (int o = 1; o < 8; ++o)
                if (h->w[o * n8 + p] != h->w[p]) ok = false;
        if (!ok) {
            delete h;
            return fail(nullptr, SN_EINVAL,
                        "sn_setup: explicit quadrature must be octant-major with octant o = "
                        "first octant mirrored by the sign bits of o, positive components and "
                        "equal weights across octants");
        }
    }
    h->ndir = (int)h->w.size();
    h->Do = h->ndir / 8;
    h->nplanes = h->nx + h->ny + h->nz - 2;

    // cross sections
    const size_t GC = (size_t)G * C;
    if (!finite_all(xs->sigt, GC) || !finite_all(xs->sigs, GC) || !finite_all(xs->q, GC) ||
        !finite_all(xs->xfer, (size_t)G * G) || (xs->psi_inc && !finite_all(xs->psi_inc, 6 * G))) {
        delete h;
        return fail(nullptr, SN_EINVAL, "sn_setup: non-finite cross section, source or inflow");
    }
    for (size_t i = 0; i < GC; ++i)
        if (xs->sigt[i] < 0 || xs->sigs[i] < 0) {
            delete h;
            return fail(nullptr, SN_EINVAL, "sn_setup: negative cross section");
        }
    if ((int64_t)G * C * 8 >= (1LL << 31)) {
        delete h;
        return fail(nullptr, SN_EINVAL, "sn_setup: ngroups * cells * 8 must stay below 2^31");
    }
    {
        // face-plane slots (4-vectors) of one plane set are indexed with 32-bit integers
        const int64_t nxy = (int64_t)h->nx * h->ny, nxz = (int64_t)h->nx * h->nz, nyz = (int64_t)h->ny * h->nz;
        const int64_t slots = 8 * std::max(nxy, std::max(nxz, nyz)) * G * (int64_t)(h->ndir / 8);
        if (slots >= (1LL << 31)) {
            delete h;
            return fail(nullptr, SN_EINVAL, "sn_setup: 8 x face cells x groups x directions per octant must stay below 2^31");
        }
    }
    if (h->Do > 128) {
        delete h;
        return fail(nullptr, SN_EINVAL, "sn_setup: at most 128 directions per octant");
    }

    // every host-side check passed: now the device
    {
        int ndev = 0;
        cudaError_t ce = cudaGetDeviceCount(&ndev);
        if (ce != cudaSuccess || ndev < 1) {
            delete h;
            return fail(nullptr, SN_ECUDA, std::string("sn_setup: no CUDA device: ") + cudaGetErrorString(ce));
        }
        cudaGetDevice(&h->dev);
    }

    sn_status s = SN_OK;
#define SN_TRY(x)               \
    do {                        \
        s = (x);                \
        if (s != SN_OK) {       \
            sn_handle hh = h;   \
            std::string m = hh->err; \
            release(hh);        \
            delete hh;          \
            return fail(nullptr, s, m); \
        }                       \
    } while (0)

    SN_TRY(dalloc(h, &h->sigt, GC));
    SN_TRY(dalloc(h, &h->sigs, GC));
    SN_TRY(dalloc(h, &h->q, GC));
    SN_TRY(dalloc(h, &h->xfer, (size_t)G * G));
    SN_TRY(dalloc(h, &h->psi_inc, 6 * (size_t)G));
    SN_TRY(upload(h, h->sigt, xs->sigt, GC));
    SN_TRY(upload(h, h->sigs, xs->sigs, GC));
    SN_TRY(upload(h, h->q, xs->q, GC));
    SN_TRY(upload(h, h->xfer, xs->xfer, (size_t)G * G));
    std::vector<double> inc(6 * G, 0.0);
    if (xs->psi_inc) inc.assign(xs->psi_inc, xs->psi_inc + 6 * G);
    SN_TRY(upload(h, h->psi_inc, inc.data(), 6 * (size_t)G));

    // direction table (first octant; the others are its mirror images)
    SN_TRY(h->fp64 ? upload_dirs<double>(h) : upload_dirs<float>(h));
    {
        std::vector<float4> da(h->Do);
        for (int d = 0; d < h->Do; ++d)
            da[d] = make_float4((float)std::fabs(h->omega[3 * d]), (float)std::fabs(h->omega[3 * d + 1]),
                                (float)std::fabs(h->omega[3 * d + 2]), 0.f);
        SN_TRY(dalloc_bytes(h, (void **)&h->dir_abs, sizeof(float4) * h->Do));
        cudaError_t e = cudaMemcpyAsync(h->dir_abs, da.data(), sizeof(float4) * h->Do, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "cudaMemcpyAsync(dir_abs)"));
    }

    // boundary inflow of one sweep: sum over faces, groups and inflowing directions
    // of w_d |Omega.n| psi_inc * area
    {
        const double area[3] = {h->ly * h->lz, h->lx * h->lz, h->lx * h->ly};
        double tot = 0.0;
        for (int g = 0; g < G; ++g)
            for (int f = 0; f < 6; ++f) {
                const double v = inc[6 * g + f];
                if (v == 0.0) continue;
                const int ax = f / 2;
                for (int d = 0; d < h->ndir; ++d) {
                    const double o = h->omega[3 * d + ax];
                    if ((f % 2 == 0 && o > 0) || (f % 2 == 1 && o < 0)) tot += h->w[d] * std::fabs(o) * v * area[ax];
                }
            }
        h->inflow = tot;
        h->inflow_box = tot;
    }

    // hyperplane table: cells (i',j',k') with i'+j'+k' = s, packed 10 bits per index
    {
        std::vector<uint32_t> cells, pos;
        hyperplane_tables(h->nx, h->ny, h->nz, h->plane_off, cells, pos);
        SN_TRY(dalloc_bytes(h, (void **)&h->plane_cells, sizeof(uint32_t) * (size_t)C));
        cudaError_t e = cudaMemcpyAsync(h->plane_cells, cells.data(), sizeof(uint32_t) * C, cudaMemcpyHostToDevice,
                                        h->stream);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "cudaMemcpyAsync(plane_cells)"));
        SN_TRY(dalloc_bytes(h, (void **)&h->plane_pos, sizeof(uint32_t) * (size_t)C));
        e = cudaMemcpyAsync(h->plane_pos, pos.data(), sizeof(uint32_t) * C, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "cudaMemcpyAsync(plane_pos)"));
    }

    // face planes: per octant, per (j',k') / (i',k') / (i',j'), per (group, direction):
    // one 4-vector of the element type
    const int64_t GD = G * h->Do;
    h->face_x = 8LL * h->ny * h->nz * GD;
    h->face_y = 8LL * h->nx * h->nz * GD;
    h->face_z = 8LL * h->nx * h->ny * GD;
    // after the planes: psi_inc of every (group, face) as a 4-vector, read by the key
    // sweep's inflow-boundary cells in place of a face slot
    h->face_in = h->face_x + h->face_y + h->face_z;
    SN_TRY(dalloc(h, &h->face, 4 * (size_t)(h->face_in + 6 * G)));
    if (!h->fp64) {
        std::vector<float> in4(24 * (size_t)G);
        for (size_t e = 0; e < in4.size(); ++e) in4[e] = (float)inc[e / 4];
        cudaError_t e = cudaMemcpyAsync(static_cast<float *>(h->face) + 4 * h->face_in, in4.data(),
                                        sizeof(float) * in4.size(), cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "cudaMemcpyAsync(inflow vectors)"));
    }
    SN_TRY(dalloc(h, &h->phi_oct, (size_t)8 * GC * 8));
    SN_TRY(dalloc(h, &h->S, GC * 8));
    SN_TRY(dalloc(h, &h->S_b, GC * 8));
    SN_TRY(dalloc(h, &h->phi_b, GC * 8));
    SN_TRY(dalloc_bytes(h, (void **)&h->acc, sizeof(double) * ACC_COUNT));
    {
        cudaError_t e = cudaMallocHost((void **)&h->acc_host, sizeof(double) * ACC_COUNT);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "cudaMallocHost"));
        e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "cudaStreamCreate"));
    }
    SN_TRY(reduce_configure(h));
    SN_TRY(build_wave(h));
    {
        // the uploads above are queued on the handle's stream (from pageable host
        // memory: staged before each call returns); the handle is complete once they land
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) SN_TRY(cuda_fail(h, e, "sn_setup: cudaStreamSynchronize"));
    }
#undef SN_TRY
    *out = h;
    return SN_OK;
}

sn_status sn_set_stream(sn_handle h, void *stream)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_set_stream: NULL handle");
    // work queued on the old stream is ordered before anything on the new one
    if (h->stream != (cudaStream_t)stream) SN_CK(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)stream;
    return SN_OK;
}

sn_status sn_get_info(sn_handle h, sn_info *info)
{
    if (!h || !info) return fail(h, SN_EINVAL, "sn_get_info: NULL argument");
    info->ncell = h->ncell;
    info->ndir = h->ndir;
    info->ngroups = h->G;
    info->nplanes = h->nplanes;
    info->dirs_per_octant = h->Do;
    info->solves_per_sweep = h->ncell * h->ndir * (int64_t)h->G;
    info->device_bytes = h->device_bytes;
    return SN_OK;
}

sn_status sn_get_quadrature(sn_handle h, double *omega, double *w)
{
    if (!h || !omega || !w) return fail(h, SN_EINVAL, "sn_get_quadrature: NULL argument");
    std::memcpy(omega, h->omega.data(), sizeof(double) * h->omega.size());
    std::memcpy(w, h->w.data(), sizeof(double) * h->w.size());
    return SN_OK;
}

sn_status sn_get_balance(sn_handle h, double *tallies)
{
    if (!h || !tallies) return fail(h, SN_EINVAL, "sn_get_balance: NULL argument");
    if (!h->tallies_valid) return fail(h, SN_ESTATE, "sn_get_balance: no sweep has run yet");
    for (int i = 0; i < 4; ++i) tallies[i] = h->tallies[i];
    return SN_OK;
}

void sn_destroy(sn_handle h)
{
    if (!h) return;
    release(h);
    delete h;
}

}  // extern "C"
