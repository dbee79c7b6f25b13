// Binned dust density (cloud-in-cell) and the adjoint of a squared-error
// loss on it: the loss of the differentiable rollout, a profile of the dust
// density like the ones the paper's test problems compare (Sec. 3).
//
// Grid: nb[k] bins of width D_k = L_k / nb[k] per axis over the box, bin
// centres at lo + (i + 1/2) D. A particle at x has s = (x - lo)/D - 1/2,
// i0 = floor(s), f = s - i0 per axis and gives its mass m to the 2^dim bins
// (i0 or i0 + 1 per axis) with the product of the weights (1 - f) and f;
// periodic axes wrap bin indices, walled axes clamp them to [0, nb - 1]
// (mass is conserved). rho_b = (deposited mass) / (bin volume).
//
// Loss L = sum_b (rho_b - target_b)^2; its gradient with respect to the
// particle positions is, per particle and axis k,
//   dL/dx_k = sum over the particle's bins of 2 (rho_b - target_b) (m / V)
//             (prod of the other axes' weights) d(weight_k)/dx_k,
// with d(1 - f)/dx = -1/D and d(f)/dx = +1/D (the weights are piecewise
// linear; the derivative is taken on the piece holding x).
//
// The deposit accumulates in binary64 with atomics, one thread per particle;
// the loss is a one-CTA reduction; the gradient a gather, one thread per
// particle.
#include "tfsph_internal.cuh"

namespace tfsph {
namespace {

constexpr int kProfThreads = 256;

struct GridArgs {
    int dim;
    int nb[3];
    int per[3];
    double lo[3];
    double inv_d[3];  // 1 / D
    double mass;
    double inv_v;     // 1 / bin volume
};

// Bin indices and weights of one particle along one axis.
template <class T>
__device__ __forceinline__ void axis_weights(const GridArgs &A, int k, T x, int idx[2], T w[2], T dw[2])
{
    const T s = (x - T(A.lo[k])) * T(A.inv_d[k]) - T(0.5);
    const T fl = floor(s);
    const T f = s - fl;
    int i0 = (int)fl;
    int i1 = i0 + 1;
    const int n = A.nb[k];
    if (A.per[k]) {
        i0 %= n;
        if (i0 < 0) i0 += n;
        i1 %= n;
        if (i1 < 0) i1 += n;
    } else {
        i0 = min(max(i0, 0), n - 1);
        i1 = min(max(i1, 0), n - 1);
    }
    idx[0] = i0;
    idx[1] = i1;
    w[0] = T(1) - f;
    w[1] = f;
    dw[0] = -T(A.inv_d[k]);
    dw[1] = T(A.inv_d[k]);
}

template <class T, int DIM>
__global__ void __launch_bounds__(kProfThreads) k_deposit(GridArgs A, const T *__restrict__ x, int64_t n,
                                                          double *__restrict__ acc)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int idx[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    T w[3][2] = {{T(1), T(0)}, {T(1), T(0)}, {T(1), T(0)}};
    T dw[3][2];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const T xk = x[(int64_t)k * n + j];
        if (!(xk == xk)) return;  // NaN: not deposited
        axis_weights(A, k, xk, idx[k], w[k], dw[k]);
    }
#pragma unroll
    for (int c = 0; c < (1 << DIM); ++c) {
        double wt = A.mass;
        int b = 0, stride = 1;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int e = (c >> k) & 1;
            wt *= (double)w[k][e];
            b += idx[k][e] * stride;
            stride *= A.nb[k];
        }
        atomicAdd(&acc[b], wt);
    }
}

// rho_b = acc_b / V in place; loss = sum (rho_b - target_b)^2 (one CTA).
__global__ void __launch_bounds__(kProfThreads) k_profile_loss(GridArgs A, int nbins, double *__restrict__ rho,
                                                               const double *__restrict__ target,
                                                               double *__restrict__ loss)
{
    __shared__ double part[kProfThreads];
    double s = 0.0;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const double r = rho[b] * A.inv_v;
        rho[b] = r;
        if (target) {
            const double d = r - target[b];
            s += d * d;
        }
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = kProfThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = part[0];
}

template <class T, int DIM>
__global__ void __launch_bounds__(kProfThreads) k_profile_grad(GridArgs A, const T *__restrict__ x, int64_t n,
                                                               const double *__restrict__ rho,
                                                               const double *__restrict__ target,
                                                               T *__restrict__ lam_x)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int idx[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    T w[3][2] = {{T(1), T(0)}, {T(1), T(0)}, {T(1), T(0)}};
    T dw[3][2] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const T xk = x[(int64_t)k * n + j];
        ok = ok && (xk == xk);
        axis_weights(A, k, xk, idx[k], w[k], dw[k]);
    }
    double g[3] = {0.0, 0.0, 0.0};
    if (ok) {
#pragma unroll
        for (int c = 0; c < (1 << DIM); ++c) {
            int b = 0, stride = 1;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                b += idx[k][(c >> k) & 1] * stride;
                stride *= A.nb[k];
            }
            const double lam = 2.0 * (rho[b] - target[b]) * A.mass * A.inv_v;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                double p = lam * (double)dw[k][(c >> k) & 1];
#pragma unroll
                for (int q = 0; q < DIM; ++q)
                    if (q != k) p *= (double)w[q][(c >> q) & 1];
                g[k] += p;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) lam_x[(int64_t)k * n + j] = T(g[k]);
}

template <class T, int DIM>
cudaError_t profile_t(const GridArgs &A, int nbins, const void *x, int64_t n, const double *target, double *rho,
                      double *loss, void *lam_x, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(rho, 0, sizeof(double) * (size_t)nbins, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + kProfThreads - 1) / kProfThreads);
    if (n > 0) k_deposit<T, DIM><<<blocks, kProfThreads, 0, s>>>(A, static_cast<const T *>(x), n, rho);
    k_profile_loss<<<1, kProfThreads, 0, s>>>(A, nbins, rho, target, loss);
    if (target && lam_x && n > 0)
        k_profile_grad<T, DIM><<<blocks, kProfThreads, 0, s>>>(A, static_cast<const T *>(x), n, rho, target,
                                                               static_cast<T *>(lam_x));
    return cudaGetLastError();
}

}  // namespace
}  // namespace tfsph

namespace {
int profile_fail(int code, const char *msg)
{
    tfsph::set_unbound_error(msg);
    return code;
}
}  // namespace

extern "C" int tfsph_dust_profile(const tfsph_grid_spec *g, const void *x, int64_t n, const void *target,
                                  void *rho, void *loss, void *lam_x, void *stream)
{
    using namespace tfsph;
    if (!g || !rho || (n > 0 && !x)) return profile_fail(TFSPH_E_INVALID_ARG, "NULL grid, x or rho");
    if (g->dim < 1 || g->dim > 3) return profile_fail(TFSPH_E_INVALID_ARG, "dim must be 1, 2 or 3");
    if (g->precision != TFSPH_FP32 && g->precision != TFSPH_FP64)
        return profile_fail(TFSPH_E_INVALID_ARG, "precision must be TFSPH_FP32 or TFSPH_FP64");
    if (n < 0 || n >= ((int64_t)1 << 40)) return profile_fail(TFSPH_E_INVALID_ARG, "n out of range");
    if (!(g->mass > 0.0) || !std::isfinite(g->mass)) return profile_fail(TFSPH_E_INVALID_ARG, "mass must be > 0");
    GridArgs A{};
    A.dim = g->dim;
    int64_t nbins = 1;
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) {
        A.nb[k] = 1;
        A.per[k] = 0;
        A.lo[k] = 0.0;
        A.inv_d[k] = 0.0;
        if (k >= g->dim) continue;
        const double L = g->hi[k] - g->lo[k];
        if (!(L > 0.0) || !std::isfinite(L)) return profile_fail(TFSPH_E_INVALID_ARG, "hi must exceed lo");
        if (g->nbins[k] < 1 || g->nbins[k] > (1 << 16))
            return profile_fail(TFSPH_E_INVALID_ARG, "nbins must be in [1, 65536] per axis");
        A.nb[k] = g->nbins[k];
        A.per[k] = g->periodic[k] ? 1 : 0;
        A.lo[k] = g->lo[k];
        A.inv_d[k] = (double)g->nbins[k] / L;
        nbins *= g->nbins[k];
        vol *= L / (double)g->nbins[k];
    }
    if (nbins > (1 << 26)) return profile_fail(TFSPH_E_INVALID_ARG, "more than 2^26 bins");
    A.mass = g->mass;
    A.inv_v = 1.0 / vol;
    if (lam_x && !target) return profile_fail(TFSPH_E_INVALID_ARG, "lam_x needs a target");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double *t = static_cast<const double *>(target);
    double *r = static_cast<double *>(rho);
    double *l = static_cast<double *>(loss);
    cudaError_t e;
    if (g->precision == TFSPH_FP64) {
        switch (g->dim) {
            case 1: e = profile_t<double, 1>(A, (int)nbins, x, n, t, r, l, lam_x, s); break;
            case 2: e = profile_t<double, 2>(A, (int)nbins, x, n, t, r, l, lam_x, s); break;
            default: e = profile_t<double, 3>(A, (int)nbins, x, n, t, r, l, lam_x, s); break;
        }
    } else {
        switch (g->dim) {
            case 1: e = profile_t<float, 1>(A, (int)nbins, x, n, t, r, l, lam_x, s); break;
            case 2: e = profile_t<float, 2>(A, (int)nbins, x, n, t, r, l, lam_x, s); break;
            default: e = profile_t<float, 3>(A, (int)nbins, x, n, t, r, l, lam_x, s); break;
        }
    }
    if (e != cudaSuccess) return profile_fail(TFSPH_E_CUDA, cudaGetErrorString(e));
    return TFSPH_OK;
}
