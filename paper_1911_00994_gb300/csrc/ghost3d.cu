// Ghost points of a sphere in the 3-D extension (include/gpmg3d.h,
// gp3_sphere_ghosts): every velocity node of the box interior with
// phi = R - |x - c| >= 0 next to a fluid node (phi < 0) is a ghost; its
// boundary point B comes from Algorithm 1 on the trilinear interpolant of
// phi on the grid's own nodes, and its row of Eq. (BCu) is the product of
// three quadratic Lagrange bases over the 27 nodes G - (k, l, m) s h.
//
// Built with -fmad=false: the march and bisection decide by the sign of
// interpolated values, so every operation is rounded on its own, in the
// order written, and the decisions are reproducible.
#include <cmath>
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/gpmg3d.h"

namespace gp3g {

constexpr int MAX_MARCH = 64;

struct Sphere {
    int N;
    double h, cx, cy, cz, R;
};

__device__ inline void node_xyz(const Sphere &S, int g, int i, int j, int k, double *p)
{
    const double ox = g == 0 ? 0.0 : 0.5, oy = g == 1 ? 0.0 : 0.5, oz = g == 2 ? 0.0 : 0.5;
    p[0] = ((double)i + ox) * S.h;
    p[1] = ((double)j + oy) * S.h;
    p[2] = ((double)k + oz) * S.h;
}

__device__ inline double phi_at(const Sphere &S, double x, double y, double z)
{
    const double dx = x - S.cx, dy = y - S.cy, dz = z - S.cz;
    return S.R - sqrt(dx * dx + dy * dy + dz * dz);
}

__device__ inline double phi_node(const Sphere &S, int g, int i, int j, int k)
{
    double p[3];
    node_xyz(S, g, i, j, k, p);
    return phi_at(S, p[0], p[1], p[2]);
}

// the box-interior positions of grid g: its own axis 1..N-1, the others 0..N-1
__device__ inline bool interior(const Sphere &S, int g, int i, int j, int k)
{
    const int c[3] = {i, j, k};
    for (int a = 0; a < 3; a++) {
        const int lo = a == g ? 1 : 0, hi = a == g ? S.N - 1 : S.N - 1;
        if (c[a] < lo || c[a] > hi) return false;
    }
    return true;
}

__device__ inline bool fluid(const Sphere &S, int g, int i, int j, int k)
{
    return interior(S, g, i, j, k) && phi_node(S, g, i, j, k) < 0.0;
}

// trilinear phi~ of grid g's own nodes at (x, y, z), cell by floor, and its gradient
__device__ inline double interp(const Sphere &S, int g, double x, double y, double z, double *gr)
{
    const double h = S.h;
    const double ox = g == 0 ? 0.0 : 0.5, oy = g == 1 ? 0.0 : 0.5, oz = g == 2 ? 0.0 : 0.5;
    const double X = x / h - ox, Y = y / h - oy, Z = z / h - oz;
    const double fi = floor(X), fj = floor(Y), fk = floor(Z);
    const int i0 = (int)fi, j0 = (int)fj, k0 = (int)fk;
    const double tx = X - fi, ty = Y - fj, tz = Z - fk;
    double f[2][2][2];  // [cz][cy][cx]
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) f[c][b][a] = phi_node(S, g, i0 + a, j0 + b, k0 + c);
    const double sx = 1.0 - tx, sy = 1.0 - ty, sz = 1.0 - tz;
    const double v00 = sx * f[0][0][0] + tx * f[0][0][1];
    const double v10 = sx * f[0][1][0] + tx * f[0][1][1];
    const double v01 = sx * f[1][0][0] + tx * f[1][0][1];
    const double v11 = sx * f[1][1][0] + tx * f[1][1][1];
    const double val = sz * (sy * v00 + ty * v10) + tz * (sy * v01 + ty * v11);
    if (gr) {
        gr[0] = (sz * (sy * (f[0][0][1] - f[0][0][0]) + ty * (f[0][1][1] - f[0][1][0])) +
                 tz * (sy * (f[1][0][1] - f[1][0][0]) + ty * (f[1][1][1] - f[1][1][0]))) / h;
        gr[1] = (sz * (sx * (f[0][1][0] - f[0][0][0]) + tx * (f[0][1][1] - f[0][0][1])) +
                 tz * (sx * (f[1][1][0] - f[1][0][0]) + tx * (f[1][1][1] - f[1][0][1]))) / h;
        gr[2] = (sy * (sx * (f[1][0][0] - f[0][0][0]) + tx * (f[1][0][1] - f[0][0][1])) +
                 ty * (sx * (f[1][1][0] - f[0][1][0]) + tx * (f[1][1][1] - f[0][1][1]))) / h;
    }
    return val;
}

__device__ inline void unit_normal(const Sphere &S, int g, const double *p, double *n)
{
    double gr[3];
    interp(S, g, p[0], p[1], p[2], gr);
    const double nn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    n[0] = gr[0] / nn;
    n[1] = gr[1] / nn;
    n[2] = gr[2] / nn;
}

__device__ inline void lagrange(double t, double *L)
{
    L[0] = (t - 1.0) * (t - 2.0) * 0.5;
    L[1] = -t * (t - 2.0);
    L[2] = t * (t - 1.0) * 0.5;
}

// one thread per slot of the u, v, w frames of the level (F = (N + 2)^3 each)
__global__ void k_sphere_ghosts(Sphere S, long long F, int cap, int *count, int *node, double *B, double *theta,
                                int *st, double *w, int *err)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 3 * F) return;
    const int g = (int)(e / F);
    const long long s = e - g * F;
    const int SN = S.N + 2;
    const int i = (int)(s % SN) - 1, j = (int)((s / SN) % SN) - 1, k = (int)(s / ((long long)SN * SN)) - 1;
    if (!interior(S, g, i, j, k) || phi_node(S, g, i, j, k) < 0.0) return;
    if (!(fluid(S, g, i + 1, j, k) || fluid(S, g, i - 1, j, k) || fluid(S, g, i, j + 1, k) ||
          fluid(S, g, i, j - 1, k) || fluid(S, g, i, j, k + 1) || fluid(S, g, i, j, k - 1)))
        return;
    const int pos = atomicAdd(count, 1);
    if (pos >= cap) {
        atomicOr(err, 1);
        return;
    }
    const double h = S.h;
    double G[3], nG[3], H[3], Hp[3], K[3], M[3];
    node_xyz(S, g, i, j, k, G);
    unit_normal(S, g, G, nG);
    for (int a = 0; a < 3; a++) M[a] = H[a] = Hp[a] = G[a];
    if (phi_node(S, g, i, j, k) != 0.0) {
        // Algorithm 1: march along -n while inside the object, then bisect
        int steps = 0;
        while (interp(S, g, H[0], H[1], H[2], nullptr) > 0.0) {
            if (steps == MAX_MARCH) {
                atomicOr(err, 2);
                break;
            }
            double n[3];
            unit_normal(S, g, H, n);
            for (int a = 0; a < 3; a++) {
                Hp[a] = H[a];
                H[a] = H[a] - 0.5 * h * n[a];
            }
            steps++;
        }
        const double dx = Hp[0] - H[0], dy = Hp[1] - H[1], dz = Hp[2] - H[2];
        const double dist = sqrt(dx * dx + dy * dy + dz * dz);
        const int nb = (int)ceil(log2(dist / (0.01 * h)));
        for (int a = 0; a < 3; a++) K[a] = M[a] = H[a];
        for (int q = 0; q < nb; q++) {
            for (int a = 0; a < 3; a++) M[a] = 0.5 * (Hp[a] + K[a]);
            if (interp(S, g, M[0], M[1], M[2], nullptr) < 0.0)
                for (int a = 0; a < 3; a++) K[a] = M[a];
            else
                for (int a = 0; a < 3; a++) Hp[a] = M[a];
        }
    }
    int sg[3];
    double th[3], L[3][3];
    for (int a = 0; a < 3; a++) {
        sg[a] = nG[a] >= 0.0 ? 1 : -1;
        th[a] = sg[a] * (G[a] - M[a]) / h;
        lagrange(th[a], L[a]);
        B[3 * pos + a] = M[a];
        theta[3 * pos + a] = th[a];
    }
    node[pos] = (int)e;
    int q = 0;
    for (int m = 0; m < 3; m++)
        for (int l = 0; l < 3; l++)
            for (int kk = 0; kk < 3; kk++, q++) {
                const int ii = i - kk * sg[0], jj = j - l * sg[1], kz = k - m * sg[2];
                const bool ok = ii >= -1 && ii <= S.N && jj >= -1 && jj <= S.N && kz >= -1 && kz <= S.N;
                if (!ok) atomicOr(err, 4);
                st[27 * pos + q] =
                    ok ? (int)(g * F + (((long long)(kz + 1) * SN + (jj + 1)) * SN + (ii + 1))) : -1;
                w[27 * pos + q] = L[0][kk] * L[1][l] * L[2][m];
            }
}

}  // namespace gp3g

extern "C" gp_status gp3_sphere_ghosts(int N, double cx, double cy, double cz, double R, int cap, int *count_dev,
                                       int *node, double *B, double *theta, int *st, double *w, int *count_host,
                                       cudaStream_t stream)
{
    if (N < 2 || N > 2048 || !(R > 0.0) || cap < 0 || !count_dev || !count_host || (cap > 0 && (!node || !B ||
        !theta || !st || !w)))
        return GP_INVALID;
    const long long S = N + 2, F = S * S * S;
    gp3g::Sphere sp{N, 1.0 / N, cx, cy, cz, R};
    cudaMemsetAsync(count_dev, 0, 2 * sizeof(int), stream);
    gp3g::k_sphere_ghosts<<<(unsigned)((3 * F + 255) / 256), 256, 0, stream>>>(sp, F, cap, count_dev, node, B, theta,
                                                                               st, w, count_dev + 1);
    int hc[2] = {0, 0};
    cudaMemcpyAsync(hc, count_dev, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GP_CUDA;
    *count_host = hc[0];
    if (hc[1]) return GP_GEOMETRY;  // capacity exceeded, march did not leave the object, or stencil off the frame
    return GP_OK;
}
