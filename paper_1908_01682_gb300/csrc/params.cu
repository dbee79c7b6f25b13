// Host-side parameter checks and the cell grid of a parameter set, shared by
// the single context and the batch.
#include <cmath>
#include <cstdio>
#include <limits>
#include <string>

#include "tfsph_internal.cuh"

namespace tfsph {

int validate_params(const tfsph_params *p, int64_t ng, int64_t nd, std::string &why)
{
    char buf[256];
    if (!p) { why = "params is NULL"; return TFSPH_E_INVALID_ARG; }
    if (p->dim < 1 || p->dim > 3) { why = "dim must be 1, 2 or 3"; return TFSPH_E_INVALID_ARG; }
    if (p->precision != TFSPH_FP32 && p->precision != TFSPH_FP64) { why = "unknown precision"; return TFSPH_E_INVALID_ARG; }
    if (p->kernel != TFSPH_KERNEL_CUBIC) { why = "unknown kernel"; return TFSPH_E_INVALID_ARG; }
    if (p->eos != TFSPH_EOS_ISOTHERMAL && p->eos != TFSPH_EOS_ADIABATIC) { why = "unknown eos"; return TFSPH_E_INVALID_ARG; }
    if (p->tstar_mode != TFSPH_TSTAR_ARITHMETIC && p->tstar_mode != TFSPH_TSTAR_HARMONIC) { why = "unknown tstar_mode"; return TFSPH_E_INVALID_ARG; }
    if (p->cell_acc != TFSPH_CELL_ACC_FP32 && p->cell_acc != TFSPH_CELL_ACC_FP64) { why = "unknown cell_acc"; return TFSPH_E_INVALID_ARG; }
    if (p->drag != TFSPH_DRAG_IDIC && p->drag != TFSPH_DRAG_ISPH && p->drag != TFSPH_DRAG_MK) { why = "unknown drag scheme"; return TFSPH_E_INVALID_ARG; }
    const double vals[] = {p->h, p->cell_size, p->m_gas, p->m_dust, p->cs, p->gamma, p->av_alpha, p->av_beta};
    for (double v : vals)
        if (!std::isfinite(v)) { why = "non-finite parameter"; return TFSPH_E_NONFINITE; }
    if (!(p->h > 0) || !(p->cell_size > 0)) { why = "h and cell_size must be > 0"; return TFSPH_E_INVALID_ARG; }
    if (!(p->m_gas > 0) || !(p->m_dust > 0)) { why = "particle masses must be > 0"; return TFSPH_E_INVALID_ARG; }
    if (!(p->cs > 0)) { why = "cs must be > 0"; return TFSPH_E_INVALID_ARG; }
    if (p->eos == TFSPH_EOS_ADIABATIC && !(p->gamma > 1.0)) { why = "gamma must be > 1"; return TFSPH_E_INVALID_ARG; }
    if (p->av_alpha < 0 || p->av_beta < 0) { why = "viscosity coefficients must be >= 0"; return TFSPH_E_INVALID_ARG; }
    if (ng < 0 || nd < 0 || ng >= (int64_t)1 << 31 || nd >= (int64_t)1 << 31) { why = "particle counts must be in [0, 2^31)"; return TFSPH_E_INVALID_ARG; }
    double ncells = 1.0;
    for (int d = 0; d < p->dim; ++d) {
        if (!std::isfinite(p->lo[d]) || !std::isfinite(p->hi[d])) { why = "non-finite box"; return TFSPH_E_NONFINITE; }
        const double L = p->hi[d] - p->lo[d];
        if (!(L > 0)) { why = "box must have hi > lo"; return TFSPH_E_INVALID_ARG; }
        if (p->periodic[d] && L < 4.0 * p->h) {
            snprintf(buf, sizeof buf, "periodic axis %d is shorter than 4h (%g < %g)", d, L, 4.0 * p->h);
            why = buf;
            return TFSPH_E_INVALID_ARG;
        }
        ncells *= fmax(1.0, floor(L / p->cell_size));
    }
    if (ncells > 1.0e9) { why = "too many cells (> 1e9); increase cell_size"; return TFSPH_E_INVALID_ARG; }
    return TFSPH_OK;
}

uint32_t cell_grid(const tfsph_params &p, int ncell[3])
{
    uint64_t nc = 1;
    for (int d = 0; d < 3; ++d) {
        ncell[d] = d < p.dim ? (int)fmax(1.0, floor((p.hi[d] - p.lo[d]) / p.cell_size)) : 1;
        nc *= (uint64_t)ncell[d];
    }
    return (uint32_t)nc;
}

namespace {

// Error-free transformations in binary64, round to nearest: s + e = a + b
// exactly (Knuth's two-sum) and p + e = a b exactly (the product's error by
// one fused multiply-add).
void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

void two_prod(double a, double b, double &p, double &e)
{
    p = a * b;
    e = std::fma(a, b, -p);
}

// Sign of (x - lo) n - i L over the reals: where x lies against the face
// between cells i - 1 and i. The six exact terms of the two-products are
// summed into a nonoverlapping expansion (Shewchuk's grow-expansion), whose
// largest nonzero component has the sign of the exact sum.
int face_sign(double x, double lo, double L, int n, int i)
{
    double t[6];
    two_prod(x, (double)n, t[0], t[1]);
    two_prod(-lo, (double)n, t[2], t[3]);
    two_prod(-(double)i, L, t[4], t[5]);
    double g[6];
    for (int k = 0; k < 6; ++k) {
        double q = t[k];
        for (int j = 0; j < k; ++j) {
            double sum, err;
            two_sum(q, g[j], sum, err);
            g[j] = err;
            q = sum;
        }
        g[k] = q;
    }
    for (int k = 5; k >= 0; --k)
        if (g[k] != 0.0) return g[k] > 0.0 ? 1 : -1;
    return 0;
}

}  // namespace

template <class T> void face_thresholds(double lo, double hi, int n, T *thr)
{
    const double L = hi - lo;
    const T inf = std::numeric_limits<T>::infinity();
    thr[0] = -inf;
    thr[n] = inf;
    for (int i = 1; i < n; ++i) {
        T f = (T)(lo + (double)i * (L / (double)n));  // within an ulp or two of the face
        // up while f lies below the face, then down while the next value below does not
        for (int k = 0; k < 64 && face_sign((double)f, lo, L, n, i) < 0; ++k) f = std::nextafter(f, inf);
        for (int k = 0; k < 64; ++k) {
            const T below = std::nextafter(f, -inf);
            if (face_sign((double)below, lo, L, n, i) < 0) break;
            f = below;
        }
        thr[i] = f;
    }
}

template void face_thresholds<float>(double, double, int, float *);
template void face_thresholds<double>(double, double, int, double *);

}  // namespace tfsph
