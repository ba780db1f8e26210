// Level-set transport for deforming bodies (Sect. 3.1): reinitialisation to a
// signed distance, Eq. (sdf), and advection of phi by a velocity field, on the
// (2N+1) x (2N+1) half-cell lattice that geometry_build reads.  One thread per
// lattice point and step; each step reads one buffer and writes the other.
//
// One-sided differences with the value beyond the lattice border equal to the
// border value; |grad phi| of Eq. (sdf) by Godunov's upwind rule (information
// leaves the zero level set); sgn(phi0) smoothed over one lattice spacing,
// phi0 / sqrt(phi0^2 + dx^2); forward Euler in the fictitious time.  The
// advection is first-order upwind.
#include <cmath>
#include <cstdio>

#include "gpmg_internal.cuh"

namespace gpmg {
namespace {

struct Diffs {
    double bx, fx, by, fy;  // backward / forward differences along x and y
};

__device__ inline Diffs diffs(const double *f, int M, int a, int b, double idx)
{
    const long long k = (long long)b * M + a;
    const double c = f[k];
    const double w = a > 0 ? f[k - 1] : c, e = a < M - 1 ? f[k + 1] : c;
    const double s = b > 0 ? f[k - M] : c, n = b < M - 1 ? f[k + M] : c;
    return Diffs{(c - w) * idx, (e - c) * idx, (c - s) * idx, (n - c) * idx};
}

__global__ void k_reinit_step(const double *phi, const double *phi0, double *out, int M, double dx, double dtau)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= M) return;
    const long long k = (long long)b * M + a;
    const double p0 = phi0[k];
    const double sg = p0 / sqrt(p0 * p0 + dx * dx);
    const Diffs D = diffs(phi, M, a, b, 1.0 / dx);
    double g2 = 0.0;
    if (sg > 0.0)
        g2 = fmax(fmax(D.bx, 0.0) * fmax(D.bx, 0.0), fmin(D.fx, 0.0) * fmin(D.fx, 0.0)) +
             fmax(fmax(D.by, 0.0) * fmax(D.by, 0.0), fmin(D.fy, 0.0) * fmin(D.fy, 0.0));
    else if (sg < 0.0)
        g2 = fmax(fmin(D.bx, 0.0) * fmin(D.bx, 0.0), fmax(D.fx, 0.0) * fmax(D.fx, 0.0)) +
             fmax(fmin(D.by, 0.0) * fmin(D.by, 0.0), fmax(D.fy, 0.0) * fmax(D.fy, 0.0));
    out[k] = phi[k] + dtau * sg * (1.0 - (sg != 0.0 ? sqrt(g2) : 0.0));
}

__global__ void k_advect_step(const double *phi, const double *wx, const double *wy, double *out, int M, double dx,
                              double dt)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= M) return;
    const long long k = (long long)b * M + a;
    const Diffs D = diffs(phi, M, a, b, 1.0 / dx);
    const double u = wx[k], v = wy[k];
    out[k] = phi[k] - dt * (fmax(u, 0.0) * D.bx + fmin(u, 0.0) * D.fx + fmax(v, 0.0) * D.by + fmin(v, 0.0) * D.fy);
}

}  // namespace

int levelset_reinit(Ctx *c, double *phi, double *work, int iters, double dtau)
{
    const int M = 2 * c->prm.N + 1;
    const double dx = 0.5 * c->prm.L / (double)c->prm.N;
    if (dtau > dx) {
        snprintf(c->msg, sizeof c->msg, "gp_levelset_reinit: dtau %.3e above the lattice spacing %.3e", dtau, dx);
        return GP_INVALID;
    }
    const size_t n = (size_t)M * M;
    double *phi0 = work, *tmp = work + n;
    cudaMemcpyAsync(phi0, phi, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    dim3 grid((M + 255) / 256, M);
    double *src = phi, *dst = tmp;
    for (int it = 0; it < iters; it++) {
        k_reinit_step<<<grid, 256, 0, c->stream>>>(src, phi0, dst, M, dx, dtau);
        double *t = src;
        src = dst;
        dst = t;
    }
    if (src != phi) cudaMemcpyAsync(phi, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    c->launches += iters;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(c->msg, sizeof c->msg, "gp_levelset_reinit: %s", cudaGetErrorString(e));
        return GP_CUDA;
    }
    return GP_OK;
}

int levelset_advect(Ctx *c, double *phi, double *work, const double *wx, const double *wy, double dt, int steps)
{
    const int M = 2 * c->prm.N + 1;
    const double dx = 0.5 * c->prm.L / (double)c->prm.N;
    const size_t n = (size_t)M * M;
    dim3 grid((M + 255) / 256, M);
    double *src = phi, *dst = work;
    for (int s = 0; s < steps; s++) {
        k_advect_step<<<grid, 256, 0, c->stream>>>(src, wx, wy, dst, M, dx, dt);
        double *t = src;
        src = dst;
        dst = t;
    }
    if (src != phi) cudaMemcpyAsync(phi, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    c->launches += steps;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(c->msg, sizeof c->msg, "gp_levelset_advect: %s", cudaGetErrorString(e));
        return GP_CUDA;
    }
    return GP_OK;
}

}  // namespace gpmg
