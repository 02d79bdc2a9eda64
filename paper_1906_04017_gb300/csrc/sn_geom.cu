// sn_geom.cu -- general hexahedral cells (the shape change of the cells of Sec. 2's
// closing remarks): the element matrices of hex.cuh for every cell of a structured
// mesh with given vertex coordinates, and the checks that keep the octant wavefront
// valid on it.
//
// Cell (i,j,k) maps the unit cube trilinearly onto its 8 vertices (node n = a + 2b +
// 4c at vertex (i+a, j+b, k+c)); trial and test functions are the same trilinear N_n
// (isoparametric Q1).  With dV = det J dxi and d_a N = sum_s adj(J)[s][a] d_s N / det J
// every integrand of M, L_a and the face matrices is a polynomial of degree <= 4 per
// reference axis, so 3-point Gauss quadrature per axis is exact; the face area vector
// of face xi_a = side is +-(dx/dxi_p x dx/dxi_q), (a, p, q) cyclic, + on side 1.
//
// The sweep keeps the structured wavefront of the box mesh: for a direction of
// octant o the inflow face of axis a is the one a box cell would have.  That holds on
// a deformed cell as long as Omega . n keeps that face's box sign everywhere on the
// face, for every direction of the quadrature: checked at the face quadrature points
// (and det J > 0 at the volume points) before the mesh is accepted.
#include <cmath>
#include <vector>

#include "hex.cuh"
#include "sn_internal.cuh"

namespace sn {

__device__ __forceinline__ void hex_shape_d(const double xi[3], double N[8], double dN[8][3])
{
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        double f[3], df[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int bit = (n >> a) & 1;
            f[a] = bit ? xi[a] : 1.0 - xi[a];
            df[a] = bit ? 1.0 : -1.0;
        }
        N[n] = f[0] * f[1] * f[2];
        dN[n][0] = df[0] * f[1] * f[2];
        dN[n][1] = f[0] * df[1] * f[2];
        dN[n][2] = f[0] * f[1] * df[2];
    }
}

// One thread per cell: element record [kHexRec] and node volumes (column sums of M)
// in the handle's element type; flag bit 0: det J <= 0 somewhere, bit 1: a face's
// Omega . n leaves its box sign for some direction.
template <typename T>
__global__ void __launch_bounds__(64) hex_elements_kernel(const double *__restrict__ xyz, int nx, int ny, int nz,
                                                          const double *__restrict__ omabs, int Do,
                                                          T *__restrict__ geom, T *__restrict__ vnode,
                                                          T *__restrict__ geomB, int *__restrict__ flag)
{
    const int64_t C = (int64_t)nx * ny * nz;
    const double g[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
        double X[8][3];
        for (int n = 0; n < 8; ++n) {
            const int64_t v = (i + (n & 1)) + (int64_t)(nx + 1) * ((j + ((n >> 1) & 1)) + (int64_t)(ny + 1) * (k + (n >> 2)));
            for (int r = 0; r < 3; ++r) X[n][r] = xyz[3 * v + r];
        }
        double M[64], L[192];
        for (int e = 0; e < 64; ++e) M[e] = 0.0;
        for (int e = 0; e < 192; ++e) L[e] = 0.0;
        int bad = 0;
        for (int i0 = 0; i0 < 3; ++i0)
            for (int i1 = 0; i1 < 3; ++i1)
                for (int i2 = 0; i2 < 3; ++i2) {
                    const double xi[3] = {g[i0], g[i1], g[i2]};
                    const double w = gw[i0] * gw[i1] * gw[i2];
                    double N[8], dN[8][3], J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                    hex_shape_d(xi, N, dN);
                    for (int n = 0; n < 8; ++n)
                        for (int r = 0; r < 3; ++r)
                            for (int s = 0; s < 3; ++s) J[r][s] += X[n][r] * dN[n][s];
                    double adj[3][3];
                    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
                    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
                    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
                    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
                    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
                    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
                    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
                    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
                    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
                    const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
                    if (!(det > 0.0)) bad |= 1;
                    for (int kk = 0; kk < 8; ++kk) {
                        double dk[3];
                        for (int a = 0; a < 3; ++a)
                            dk[a] = adj[0][a] * dN[kk][0] + adj[1][a] * dN[kk][1] + adj[2][a] * dN[kk][2];
                        for (int jj = 0; jj < 8; ++jj) {
                            M[8 * kk + jj] += w * det * N[kk] * N[jj];
                            for (int a = 0; a < 3; ++a) L[64 * a + 8 * kk + jj] -= w * N[jj] * dk[a];
                        }
                    }
                }
        T *out = geom + c * kHexRec;
        for (int e = 0; e < 64; ++e) out[kHexM + e] = (T)M[e];
        for (int e = 0; e < 192; ++e) out[kHexL + e] = (T)L[e];
        // B of every octant starts from L (the outflow faces are added below)
        double Bo[8][kHexB];
        for (int o = 0; o < 8; ++o)
            for (int e = 0; e < kHexB; ++e) Bo[o][e] = L[e];
        auto L2B = [&](int o, int cc, int k2, int j2) -> double & { return Bo[o][64 * cc + 8 * k2 + j2]; };
        for (int n = 0; n < 8; ++n) {
            double s = 0.0;
            for (int kk = 0; kk < 8; ++kk) s += M[8 * kk + n];
            vnode[c * 8 + n] = (T)s;
        }
        for (int f = 0; f < 6; ++f) {
            const int a = f / 2, side = f % 2, p = (a + 1) % 3, q = (a + 2) % 3;
            int fn[4];
            for (int t = 0; t < 4; ++t) {
                const int lo = t & 1, hi = t >> 1;
                fn[t] = a == 0 ? side + 2 * lo + 4 * hi : (a == 1 ? lo + 2 * side + 4 * hi : lo + 2 * hi + 4 * side);
            }
            double F[3][16];
            for (int e = 0; e < 48; ++e) F[e / 16][e % 16] = 0.0;
            for (int ip = 0; ip < 3; ++ip)
                for (int iq = 0; iq < 3; ++iq) {
                    double xi[3];
                    xi[a] = side;
                    xi[p] = g[ip];
                    xi[q] = g[iq];
                    const double w = gw[ip] * gw[iq];
                    double N[8], dN[8][3], tp[3] = {0, 0, 0}, tq[3] = {0, 0, 0};
                    hex_shape_d(xi, N, dN);
                    for (int n = 0; n < 8; ++n)
                        for (int r = 0; r < 3; ++r) {
                            tp[r] += X[n][r] * dN[n][p];
                            tq[r] += X[n][r] * dN[n][q];
                        }
                    const double sg = side ? 1.0 : -1.0;
                    const double av[3] = {sg * (tp[1] * tq[2] - tp[2] * tq[1]), sg * (tp[2] * tq[0] - tp[0] * tq[2]),
                                          sg * (tp[0] * tq[1] - tp[1] * tq[0])};
                    for (int cc = 0; cc < 3; ++cc)
                        for (int t = 0; t < 4; ++t)
                            for (int u = 0; u < 4; ++u) F[cc][4 * t + u] += w * av[cc] * N[fn[t]] * N[fn[u]];
                    // the face keeps its box sign of Omega . n for every direction
                    for (int o = 0; o < 8; ++o)
                        for (int d = 0; d < Do; ++d) {
                            double dot = 0.0;
                            for (int cc = 0; cc < 3; ++cc)
                                dot += ((o >> cc) & 1 ? -1.0 : 1.0) * omabs[3 * d + cc] * av[cc];
                            const bool outflow = (side == 1) == !((o >> a) & 1);
                            if (outflow ? dot < 0.0 : dot > 0.0) bad |= 2;
                        }
                }
            for (int cc = 0; cc < 3; ++cc)
                for (int e = 0; e < 16; ++e) out[kHexF + f * 48 + cc * 16 + e] = (T)F[cc][e];
            // this face is the outflow face of axis a in the octants whose bit a is
            // 1 - side: add it into their B (from the FP64 values)
            for (int o = 0; o < 8; ++o) {
                if (((o >> a) & 1) != 1 - side) continue;
                for (int cc = 0; cc < 3; ++cc)
                    for (int t = 0; t < 4; ++t)
                        for (int u = 0; u < 4; ++u) L2B(o, cc, fn[t], fn[u]) += F[cc][4 * t + u];
            }
        }
        for (int o = 0; o < 8; ++o)
            for (int e = 0; e < kHexB; ++e) geomB[(c * 8 + o) * kHexB + e] = (T)Bo[o][e];
        if (bad) atomicOr(flag, bad);
    }
}

template <typename T>
static sn_status build_geometry(sn_handle h, const double *xyz_host, void **geom, void **vnode, void **omabs,
                                void **geomB)
{
    const int64_t C = h->ncell, NV = (int64_t)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
    double *dxyz = nullptr, *dom = nullptr;
    int *dflag = nullptr;
    std::vector<double> om(3 * (size_t)h->Do);
    for (int d = 0; d < h->Do; ++d)
        for (int r = 0; r < 3; ++r) om[3 * d + r] = std::fabs(h->omega[3 * d + r]);
    std::vector<T> omT(om.begin(), om.end());
    cudaError_t e = cudaMalloc(&dxyz, sizeof(double) * 3 * NV);
    if (e == cudaSuccess) e = cudaMalloc(&dom, sizeof(double) * om.size());
    if (e == cudaSuccess) e = cudaMalloc(&dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(geom, sizeof(T) * C * kHexRec);
    if (e == cudaSuccess) e = cudaMalloc(vnode, sizeof(T) * C * 8);
    if (e == cudaSuccess) e = cudaMalloc(omabs, sizeof(T) * omT.size());
    if (e == cudaSuccess) e = cudaMalloc(geomB, sizeof(T) * C * 8 * kHexB);
    cudaStream_t st = h->stream;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dxyz, xyz_host, sizeof(double) * 3 * NV, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dom, om.data(), sizeof(double) * om.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*omabs, omT.data(), sizeof(T) * omT.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(int), st);
    int flag = 0;
    if (e == cudaSuccess) {
        int64_t grid = (C + 63) / 64;
        if (grid > (int64_t)num_sms() * 32) grid = (int64_t)num_sms() * 32;
        hex_elements_kernel<T><<<(unsigned)grid, 64, 0, st>>>(dxyz, h->nx, h->ny, h->nz, dom, h->Do, (T *)*geom,
                                                              (T *)*vnode, (T *)*geomB, dflag);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    // the element kernel and the flag are complete before the scratch buffers go
    {
        const cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
    }
    cudaFree(dxyz);
    cudaFree(dom);
    cudaFree(dflag);
    if (e != cudaSuccess) return cuda_fail(h, e, "sn_set_geometry");
    if (flag & 1) return fail(h, SN_EINVAL, "sn_set_geometry: a cell has a non-positive Jacobian");
    if (flag & 2)
        return fail(h, SN_EINVAL, "sn_set_geometry: a face changes its inflow/outflow side for some direction "
                                  "(mesh too deformed for the structured sweep)");
    return SN_OK;
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_set_geometry(sn_handle h, const double *xyz)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_set_geometry: NULL handle");
    if (h->K > 1) return fail(h, SN_EINVAL, "sn_set_geometry: not with anisotropic scattering");
    SN_CK(h, cudaStreamSynchronize(h->stream));
    auto release = [h]() {
        void *b[] = {h->geom, h->vnode, h->omabs, h->geomB};
        for (void *p : b)
            if (p) cudaFree(p);
        h->geom = h->vnode = h->omabs = h->geomB = nullptr;
    };
    if (!xyz) {
        release();
        h->inflow = h->inflow_box;
        return SN_OK;
    }
    const int64_t NV = (int64_t)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
    for (int64_t i = 0; i < 3 * NV; ++i)
        if (!std::isfinite(xyz[i])) return fail(h, SN_EINVAL, "sn_set_geometry: non-finite vertex coordinate");
    void *geom = nullptr, *vnode = nullptr, *omabs = nullptr, *geomB = nullptr;
    sn_status s = h->fp64 ? build_geometry<double>(h, xyz, &geom, &vnode, &omabs, &geomB)
                          : build_geometry<float>(h, xyz, &geom, &vnode, &omabs, &geomB);
    if (s != SN_OK) {
        void *b[] = {geom, vnode, omabs, geomB};
        for (void *p : b)
            if (p) cudaFree(p);
        return s;
    }
    release();
    h->geom = geom;
    h->vnode = vnode;
    h->omabs = omabs;
    h->geomB = geomB;
    // boundary inflow of one sweep: the inflow planes' outward area vectors (sum of
    // the boundary faces' bilinear patches, half the cross product of the diagonals)
    const int nx = h->nx, ny = h->ny, nz = h->nz;
    auto V = [&](int i, int j, int k) { return xyz + 3 * ((int64_t)i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k)); };
    double area[6][3] = {{0}};
    auto add_patch = [&](int f, const double *p00, const double *p10, const double *p11, const double *p01) {
        const double d1[3] = {p11[0] - p00[0], p11[1] - p00[1], p11[2] - p00[2]};
        const double d2[3] = {p01[0] - p10[0], p01[1] - p10[1], p01[2] - p10[2]};
        const double cr[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
        // outward: the component along the plane's axis has the side's sign (the
        // checks above keep every face close enough to its box orientation)
        const int ax = f / 2;
        const double sg = ((f % 2) ? 1.0 : -1.0) * (cr[ax] >= 0.0 ? 0.5 : -0.5);
        for (int r = 0; r < 3; ++r) area[f][r] += sg * cr[r];
    };
    for (int side = 0; side < 2; ++side) {
        const int i = side ? nx : 0, j = side ? ny : 0, k = side ? nz : 0;
        for (int b = 0; b < nz; ++b)
            for (int a = 0; a < ny; ++a) add_patch(0 + side, V(i, a, b), V(i, a + 1, b), V(i, a + 1, b + 1), V(i, a, b + 1));
        for (int b = 0; b < nx; ++b)
            for (int a = 0; a < nz; ++a) add_patch(2 + side, V(b, j, a), V(b, j, a + 1), V(b + 1, j, a + 1), V(b + 1, j, a));
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) add_patch(4 + side, V(a, b, k), V(a + 1, b, k), V(a + 1, b + 1, k), V(a, b + 1, k));
    }
    std::vector<double> inc(6 * (size_t)h->G);
    if (h->fp64) {
        SN_CK(h, cudaMemcpyAsync(inc.data(), h->psi_inc, sizeof(double) * inc.size(), cudaMemcpyDeviceToHost, h->stream));
        SN_CK(h, cudaStreamSynchronize(h->stream));
    } else {
        std::vector<float> f32(inc.size());
        SN_CK(h, cudaMemcpyAsync(f32.data(), h->psi_inc, sizeof(float) * f32.size(), cudaMemcpyDeviceToHost, h->stream));
        SN_CK(h, cudaStreamSynchronize(h->stream));
        for (size_t i = 0; i < f32.size(); ++i) inc[i] = f32[i];
    }
    double tot = 0.0;
    for (int g = 0; g < h->G; ++g)
        for (int f = 0; f < 6; ++f) {
            if (inc[6 * g + f] == 0.0) continue;
            const int ax = f / 2;
            for (int d = 0; d < h->ndir; ++d) {
                const double *o = &h->omega[3 * d];
                if ((f % 2 == 0 && o[ax] > 0) || (f % 2 == 1 && o[ax] < 0)) {
                    const double on = o[0] * area[f][0] + o[1] * area[f][1] + o[2] * area[f][2];
                    tot += h->w[d] * (-on) * inc[6 * g + f];
                }
            }
        }
    h->inflow = tot;
    for (int p = 0; p < 2; ++p)
        if (h->graphs.exec[p]) { cudaGraphExecDestroy(h->graphs.exec[p]); h->graphs.exec[p] = nullptr; }
    h->graphs.phi_user = nullptr;
    h->tallies_valid = false;
    return SN_OK;
}

}  // extern "C"
