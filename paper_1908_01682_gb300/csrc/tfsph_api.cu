// C ABI of libtfsph: context set-up, the step sequence, field export.
//
// Step sequence on the context's stream (no host synchronisation):
//   [bin]     count -> scan (3 launches) -> scatter -> rank+gather   (bin.cu)
//   [density] gas summation density and p/rho^2                       (sph.cu)
//   [force]   gas pressure (+ viscous) acceleration, de/dt             (sph.cu)
//   [drag]    per-cell implicit drag, particle update, next keys       (drag.cu)
// The first two form "prepare" and are skipped when a field export has
// already binned the current positions.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tfsph_internal.cuh"

using namespace tfsph;

struct tfsph_ctx {
    tfsph_params p{};
    int precision = TFSPH_FP32;
    int dim = 1;
    int cell_acc = TFSPH_CELL_ACC_FP64;
    size_t tsize = 4;
    cudaStream_t stream = nullptr;
    int device = 0;
    int ncell[3] = {1, 1, 1};
    int reach[3] = {0, 0, 0};
    uint32_t ncells = 1;
    PhaseBufs G, D;
    void *rho_g = nullptr;
    void *rho_d = nullptr;
    void *acc = nullptr;
    uint32_t *bsum = nullptr;
    int64_t nblk = 1;
    void *partials = nullptr;
    int npart = 1;
    void *scalar = nullptr;
    int *d_err = nullptr;
    int *d_flags = nullptr;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    // adjoint scratch (allocated by the first tfsph_step_adjoint)
    void *adj_gx4 = nullptr, *adj_gv4 = nullptr, *adj_dx4 = nullptr, *adj_du4 = nullptr;
    void *adj_lA = nullptr, *adj_out = nullptr, *adj_lrho = nullptr, *adj_lts = nullptr;
    void *adj_host = nullptr;  // device mirror of host adjoint arrays
    alignas(64) unsigned char geo[sizeof(Geo<double>)];
    alignas(64) unsigned char phys[sizeof(Phys<double>)];
    NbList nbl;                 // gas neighbour list of the density pass (nbl.idx null: none)
    XDragBufs xb;               // per-particle scratch of the ISPH / MK drag
    bool nbl_valid = false;     // nbl belongs to the current binning
    bool prepared = false;      // binning and density of the current state are done
    bool forced = false;        // ... and acc holds its pressure acceleration
    bool counts_dirty = false;  // a binning did not finish: zero the cell counts first
    bool has_frozen = false;
    int64_t steps = 0;
    int64_t device_bytes = 0;
    int64_t launches = 0;
    // phase timing: one set of TFSPH_PROF_NPHASE + 1 events per profiled step
    bool profiling = false;
    std::vector<std::vector<cudaEvent_t>> prof_sets;
    size_t prof_used = 0;
    double prof_ms[TFSPH_PROF_NPHASE] = {0};
    int64_t prof_steps = 0;
    int64_t prof_launches = 0;
    std::vector<void *> allocs;
    std::string err;
};

namespace {

thread_local std::string g_init_error;

int fail(tfsph_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_init_error = msg;
    return code;
}

int cuda_fail(tfsph_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? TFSPH_E_OOM : TFSPH_E_CUDA, m);
}

#define TF_CUDA(c, call)                                        \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
    } while (0)

int dalloc(tfsph_ctx *c, void **out, size_t bytes)
{
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(c, e, "cudaMalloc");
    }
    c->allocs.push_back(*out);
    c->device_bytes += (int64_t)bytes;
    return TFSPH_OK;
}

template <class T> void build_geo(tfsph_ctx *c)
{
    Geo<T> G{};
    Phys<T> Ph{};
    make_geo_phys<T>(c->p, c->ncell, c->ncells, G, Ph);
    for (int d = 0; d < 3; ++d) c->reach[d] = G.R[d];
    memcpy(c->geo, &G, sizeof(G));
    memcpy(c->phys, &Ph, sizeof(Ph));
}

// Device table of the exact cell-face thresholds of every axis (cell_key);
// the geometry's per-axis pointers are set into it.
template <class T> int upload_thresholds(tfsph_ctx *c)
{
    Geo<T> &G = *reinterpret_cast<Geo<T> *>(c->geo);
    size_t off[3] = {0, 0, 0}, total = 0;
    for (int d = 0; d < c->dim; ++d) {
        off[d] = total;
        total += (size_t)G.n[d] + 1;
    }
    std::vector<T> h(total);
    for (int d = 0; d < c->dim; ++d) face_thresholds<T>(c->p.lo[d], c->p.hi[d], G.n[d], h.data() + off[d]);
    void *dev = nullptr;
    int rc = dalloc(c, &dev, total * sizeof(T));
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(dev, h.data(), total * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
    for (int d = 0; d < c->dim; ++d) G.thr[d] = static_cast<const T *>(dev) + off[d];
    return TFSPH_OK;
}

LaunchCtx lctx(const tfsph_ctx *c)
{
    LaunchCtx L;
    L.stream = c->stream;
    L.precision = c->precision;
    L.dim = c->dim;
    L.d_err = c->d_err;
    L.ev = nullptr;
    return L;
}

// Device address of a page-locked (registered) host buffer, through which
// kernels read or write it directly over the host link; NULL for pageable
// memory, which goes through the staging buffer.
void *mapped_host(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

// Device copies of user arrays: returns device pointers (host input is
// staged, unless every array is page-locked: then kernels read it in place
// and *staged stays false).
int stage_inputs(tfsph_ctx *c, const void *const *arrs, int narr, int64_t n, const uint8_t *frozen, int mem_kind,
                 std::vector<const void *> &dev, const uint8_t **dev_frozen, bool *staged = nullptr)
{
    dev.assign(narr, nullptr);
    *dev_frozen = nullptr;
    if (staged) *staged = false;
    if (n == 0) return TFSPH_OK;
    for (int k = 0; k < narr; ++k)
        if (!arrs[k]) return fail(c, TFSPH_E_INVALID_ARG, "NULL input array");
    if (mem_kind == TFSPH_MEM_HOST) {
        std::vector<const void *> mapped(narr, nullptr);
        bool all = true;
        for (int k = 0; k < narr && all; ++k) all = (mapped[k] = mapped_host(arrs[k])) != nullptr;
        const uint8_t *mf = nullptr;
        if (all && frozen) all = (mf = static_cast<const uint8_t *>(mapped_host(frozen))) != nullptr;
        if (all) {
            dev = mapped;
            *dev_frozen = mf;
            return TFSPH_OK;
        }
    }
    if (mem_kind == TFSPH_MEM_DEVICE) {
        for (int k = 0; k < narr; ++k) dev[k] = arrs[k];
        *dev_frozen = frozen;
        return TFSPH_OK;
    }
    const size_t need = (size_t)narr * (size_t)n * c->tsize + (frozen ? (size_t)n + 256 : 0);
    if (need > c->staging_bytes) return fail(c, TFSPH_E_INTERNAL, "staging buffer too small");
    if (staged) *staged = true;
    char *base = static_cast<char *>(c->staging);
    for (int k = 0; k < narr; ++k) {
        char *dst = base + (size_t)k * (size_t)n * c->tsize;
        TF_CUDA(c, cudaMemcpyAsync(dst, arrs[k], (size_t)n * c->tsize, cudaMemcpyHostToDevice, c->stream));
        dev[k] = dst;
    }
    if (frozen) {
        char *dst = base + (size_t)narr * (size_t)n * c->tsize;
        TF_CUDA(c, cudaMemcpyAsync(dst, frozen, (size_t)n, cudaMemcpyHostToDevice, c->stream));
        *dev_frozen = reinterpret_cast<const uint8_t *>(dst);
    }
    return TFSPH_OK;
}

// Loads a full particle state, computes keys and checks it (synchronises).
int load_state(tfsph_ctx *c, const void *const *gas, const void *const *dust, const uint8_t *frozen, int mem_kind)
{
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
    if ((c->G.n > 0 && !gas) || (c->D.n > 0 && !dust)) return fail(c, TFSPH_E_INVALID_ARG, "NULL array list");
    const int d = c->dim;
    const int ngas_arr = 2 * d + (c->p.eos == TFSPH_EOS_ADIABATIC ? 1 : 0);
    const int ndust_arr = 2 * d + 1;
    LaunchCtx L = lctx(c);
    std::vector<const void *> dv;
    const uint8_t *dfz = nullptr;
    bool staged = false;
    int rc = stage_inputs(c, gas, ngas_arr, c->G.n, frozen, mem_kind, dv, &dfz, &staged);
    if (rc) return rc;
    c->G.cur = 0;
    TF_CUDA(c, launch_pack(L, c->G, dv.data(), c->p.eos == TFSPH_EOS_ADIABATIC, dfz, true));
    // the gas staging area is reused for dust only after the pack has consumed it
    if (staged) TF_CUDA(c, cudaStreamSynchronize(c->stream));
    rc = stage_inputs(c, dust, ndust_arr, c->D.n, nullptr, mem_kind, dv, &dfz);
    if (rc) return rc;
    c->D.cur = 0;
    TF_CUDA(c, launch_pack(L, c->D, dv.data(), 1, nullptr, false));
    TF_CUDA(c, launch_keys(L, c->geo, c->G));
    TF_CUDA(c, launch_keys(L, c->geo, c->D));
    TF_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
    TF_CUDA(c, launch_check(L, c->geo, c->G, 1, c->d_flags));
    TF_CUDA(c, launch_check(L, c->geo, c->D, 0, c->d_flags));
    int flags = 0;
    TF_CUDA(c, cudaMemcpyAsync(&flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TF_CUDA(c, cudaStreamSynchronize(c->stream));
    if (flags & 1) return fail(c, TFSPH_E_NONFINITE, "non-finite position, velocity or energy in the input");
    if (flags & 4) return fail(c, TFSPH_E_NONFINITE, "dust t_stop must be finite and > 0");
    if (flags & 2) return fail(c, TFSPH_E_OUT_OF_DOMAIN, "a moving particle lies outside [lo, hi)");
    bool any_frozen = false;
    if (frozen && c->G.n > 0) {
        if (mem_kind == TFSPH_MEM_HOST) {
            const uint8_t *f = frozen;
            for (int64_t i = 0; i < c->G.n && !any_frozen; ++i) any_frozen = f[i] != 0;
        } else {
            any_frozen = true;  // device flags: assume present (only costs an id read per particle)
        }
    }
    c->has_frozen = any_frozen;
    c->prepared = false;
    c->forced = false;
    c->nbl_valid = false;
    c->steps = 0;
    return TFSPH_OK;
}

int fold_profile(tfsph_ctx *c)
{
    if (c->prof_used == 0) return TFSPH_OK;
    TF_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < c->prof_used; ++k) {
        auto &ev = c->prof_sets[k];
        for (int ph = 0; ph < TFSPH_PROF_NPHASE; ++ph) {
            float ms = 0.f;
            TF_CUDA(c, cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]));
            c->prof_ms[ph] += ms;
        }
    }
    c->prof_used = 0;
    return TFSPH_OK;
}

// Events for the next profiled step (NULL when not profiling).
int next_events(tfsph_ctx *c, cudaEvent_t **out)
{
    *out = nullptr;
    if (!c->profiling) return TFSPH_OK;
    if (c->prof_used == 64) {
        int rc = fold_profile(c);
        if (rc) return rc;
    }
    if (c->prof_used == c->prof_sets.size()) {
        std::vector<cudaEvent_t> ev(TFSPH_PROF_NPHASE + 1);
        for (auto &e : ev) TF_CUDA(c, cudaEventCreate(&e));
        c->prof_sets.push_back(ev);
    }
    *out = c->prof_sets[c->prof_used++].data();
    return TFSPH_OK;
}

int prepare(tfsph_ctx *c, cudaEvent_t *ev = nullptr)
{
    if (c->prepared) {
        if (ev)
            for (int k = 1; k <= TFSPH_PROF_DENSITY + 1; ++k) TF_CUDA(c, cudaEventRecord(ev[k], c->stream));
        return TFSPH_OK;
    }
    LaunchCtx L = lctx(c);
    L.ev = ev;
    if (c->counts_dirty) {
        TF_CUDA(c, cudaMemsetAsync(c->G.count, 0, (size_t)c->ncells * 4, c->stream));
        TF_CUDA(c, cudaMemsetAsync(c->D.count, 0, (size_t)c->ncells * 4, c->stream));
    }
    c->counts_dirty = true;
    TF_CUDA(c, launch_bin(L, c->geo, c->G, c->D, c->bsum, c->nblk));
    c->counts_dirty = false;
    c->launches += (c->G.n + c->D.n > 0) ? 6 : 3;
    TF_CUDA(c, launch_density(L, c->geo, c->phys, c->G, c->rho_g, true, nullptr, nullptr,
                              c->nbl.idx ? &c->nbl : nullptr));
    c->nbl_valid = c->nbl.idx != nullptr;
    if (c->G.n > 0) c->launches += 1;
    if (ev) TF_CUDA(c, cudaEventRecord(ev[TFSPH_PROF_DENSITY + 1], c->stream));
    c->prepared = true;
    return TFSPH_OK;
}

// Binning, density and pressure acceleration of the current state (what the
// step and its adjoint both start from); done once per state.
int forward_quantities(tfsph_ctx *c, cudaEvent_t *ev = nullptr)
{
    int rc = prepare(c, ev);
    if (rc) return rc;
    if (c->G.n > 0 && !c->forced) {
        LaunchCtx L = lctx(c);
        TF_CUDA(c, launch_force(L, c->geo, c->phys, c->G, c->rho_g, c->acc, c->nbl_valid ? &c->nbl : nullptr));
        c->launches += 1;
    }
    c->forced = true;
    if (ev) TF_CUDA(c, cudaEventRecord(ev[TFSPH_PROF_FORCE + 1], c->stream));
    return TFSPH_OK;
}

__global__ void k_mask_ids(const uint32_t *__restrict__ id, int n, uint32_t *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = id[i] & kIdMask;
}

// Copies `bytes` from device `src` to `out` (host or device), synchronising for host.
int emit(tfsph_ctx *c, const void *src, size_t bytes, void *out, int mem_kind)
{
    if (bytes == 0) return TFSPH_OK;
    if (mem_kind == TFSPH_MEM_DEVICE) {
        if (src != out) TF_CUDA(c, cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return TFSPH_OK;
    }
    TF_CUDA(c, cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    TF_CUDA(c, cudaStreamSynchronize(c->stream));
    return TFSPH_OK;
}

}  // namespace

void tfsph::set_unbound_error(const char *msg) { g_init_error = msg; }

extern "C" {

int tfsph_version(void) { return 10000; }

const char *tfsph_status_string(int code)
{
    switch (code) {
        case TFSPH_OK: return "TFSPH_OK";
        case TFSPH_E_INVALID_ARG: return "TFSPH_E_INVALID_ARG";
        case TFSPH_E_NONFINITE: return "TFSPH_E_NONFINITE";
        case TFSPH_E_OUT_OF_DOMAIN: return "TFSPH_E_OUT_OF_DOMAIN";
        case TFSPH_E_CUDA: return "TFSPH_E_CUDA";
        case TFSPH_E_OOM: return "TFSPH_E_OOM";
        case TFSPH_E_INTERNAL: return "TFSPH_E_INTERNAL";
        case TFSPH_E_TIMEOUT: return "TFSPH_E_TIMEOUT";
        default: return "TFSPH_E_UNKNOWN";
    }
}

const char *tfsph_last_error(const tfsph_ctx *c) { return c ? c->err.c_str() : g_init_error.c_str(); }

void tfsph_destroy(tfsph_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto &set : c->prof_sets)
        for (cudaEvent_t e : set) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

int tfsph_init(tfsph_ctx **out, const tfsph_params *p, const void *const *gas, int64_t n_gas,
               const void *const *dust, int64_t n_dust, const uint8_t *frozen, int mem_kind)
{
    if (!out) return fail(nullptr, TFSPH_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    int rc = validate_params(p, n_gas, n_dust, why);
    if (rc) return fail(nullptr, rc, why);
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(nullptr, TFSPH_E_INVALID_ARG, "bad mem_kind");
    if ((n_gas > 0 && !gas) || (n_dust > 0 && !dust)) return fail(nullptr, TFSPH_E_INVALID_ARG, "NULL array list");

    tfsph_ctx *c = new (std::nothrow) tfsph_ctx();
    if (!c) return fail(nullptr, TFSPH_E_OOM, "host allocation failed");
    c->p = *p;
    c->precision = p->precision;
    c->dim = p->dim;
    c->cell_acc = p->precision == TFSPH_FP64 ? TFSPH_CELL_ACC_FP64 : p->cell_acc;
    c->tsize = p->precision == TFSPH_FP64 ? 8 : 4;
    c->ncells = cell_grid(*p, c->ncell);
    c->G.n = n_gas;
    c->D.n = n_dust;
    if (p->precision == TFSPH_FP64) build_geo<double>(c);
    else build_geo<float>(c);

    auto bail = [&](int code) {
        std::string m = c->err;
        tfsph_destroy(c);
        g_init_error = m;
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));

    if ((rc = p->precision == TFSPH_FP64 ? upload_thresholds<double>(c) : upload_thresholds<float>(c)))
        return bail(rc);
    const size_t v4 = 4 * c->tsize;
    PhaseBufs *ph[2] = {&c->G, &c->D};
    for (PhaseBufs *P : ph) {
        const size_t n = (size_t)P->n;
        void *tmp;
        for (int b = 0; b < 2; ++b) {
            if ((rc = dalloc(c, &P->pos[b], n * v4))) return bail(rc);
            if ((rc = dalloc(c, &P->vel[b], n * v4))) return bail(rc);
            if ((rc = dalloc(c, &tmp, n * 4))) return bail(rc);
            P->id[b] = static_cast<uint32_t *>(tmp);
        }
        if ((rc = dalloc(c, &tmp, n * 4))) return bail(rc);
        P->key = static_cast<uint32_t *>(tmp);
        if ((rc = dalloc(c, &tmp, n * 4))) return bail(rc);
        P->tmp_src = static_cast<uint32_t *>(tmp);
        if ((rc = dalloc(c, &tmp, n * 4))) return bail(rc);
        P->tmp_id = static_cast<uint32_t *>(tmp);
        if ((rc = dalloc(c, &tmp, (size_t)c->ncells * 4))) return bail(rc);
        P->count = static_cast<uint32_t *>(tmp);
        if ((rc = dalloc(c, &tmp, ((size_t)c->ncells + 1) * 4))) return bail(rc);
        P->start = static_cast<uint32_t *>(tmp);
        e = cudaMemset(P->count, 0, (size_t)c->ncells * 4);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemset"));
    }
    if ((rc = dalloc(c, &c->rho_g, (size_t)n_gas * c->tsize))) return bail(rc);
    if ((rc = dalloc(c, &c->rho_d, (size_t)n_dust * c->tsize))) return bail(rc);
    if ((rc = dalloc(c, &c->acc, (size_t)n_gas * v4))) return bail(rc);
    // neighbour list of the gas pair sums (skipped when it would not pay or fit)
    {
        int cap = 0, oc = 0;
        int64_t tiles = 0;
        if (nblist_layout(c->geo, c->precision, c->dim, n_gas, &cap, &oc, &tiles)) {
            // cap / 4 groups of four entries per tile plus one spare group
            const size_t bytes = (size_t)tiles * (size_t)(cap / 4 + 1) * (size_t)oc * 8;
            if (bytes <= ((size_t)16 << 30)) {
                void *tmp0 = nullptr;
                if ((rc = dalloc(c, &tmp0, bytes))) return bail(rc);
                c->nbl.idx = static_cast<unsigned long long *>(tmp0);
                if ((rc = dalloc(c, &tmp0, (size_t)tiles * (size_t)oc * 2))) return bail(rc);
                c->nbl.cnt = static_cast<uint16_t *>(tmp0);
                c->nbl.cap = cap;
                c->nbl.owned_cap = oc;
            }
        }
    }
    if (p->drag != TFSPH_DRAG_IDIC) {
        if ((rc = dalloc(c, &c->xb.g4, (size_t)n_gas * v4))) return bail(rc);
        if ((rc = dalloc(c, &c->xb.g1, (size_t)n_gas * c->tsize))) return bail(rc);
        if ((rc = dalloc(c, &c->xb.d4, (size_t)n_dust * v4))) return bail(rc);
        if ((rc = dalloc(c, &c->xb.d4b, (size_t)n_dust * v4))) return bail(rc);
    }
    c->nblk = ((int64_t)c->ncells + kScanTile - 1) / kScanTile;
    void *tmp;
    if ((rc = dalloc(c, &tmp, (size_t)c->nblk * 2 * 4))) return bail(rc);
    c->bsum = static_cast<uint32_t *>(tmp);
    c->npart = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (n_gas + 255) / 256));
    if ((rc = dalloc(c, &c->partials, (size_t)c->npart * c->tsize))) return bail(rc);
    if ((rc = dalloc(c, &c->scalar, 64))) return bail(rc);
    if ((rc = dalloc(c, &tmp, 64))) return bail(rc);
    c->d_err = static_cast<int *>(tmp);
    if ((rc = dalloc(c, &tmp, 64))) return bail(rc);
    c->d_flags = static_cast<int *>(tmp);
    e = cudaMemset(c->d_err, 0, 64);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemset"));
    // staging for host I/O: the larger phase's input arrays (+ frozen flags), or a field export
    const int64_t nmax = std::max<int64_t>(n_gas, n_dust);
    const size_t stage = std::max<size_t>((size_t)(2 * p->dim + 1) * (size_t)nmax * c->tsize + (size_t)n_gas + 256,
                                          ((size_t)c->ncells + 1) * 4 + 256);
    if ((rc = dalloc(c, &c->staging, std::max<size_t>(stage, (size_t)nmax * 8 + 256)))) return bail(rc);
    c->staging_bytes = std::max<size_t>(stage, (size_t)nmax * 8 + 256);

    rc = load_state(c, gas, dust, frozen, mem_kind);
    if (rc) return bail(rc);
    *out = c;
    return TFSPH_OK;
}

int tfsph_set_state(tfsph_ctx *c, const void *const *gas, const void *const *dust, const uint8_t *frozen,
                    int mem_kind)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    return load_state(c, gas, dust, frozen, mem_kind);
}

int tfsph_set_stream(tfsph_ctx *c, void *stream)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    c->stream = static_cast<cudaStream_t>(stream);
    return TFSPH_OK;
}

int tfsph_step(tfsph_ctx *c, double tau, const void *t_stop, int mem_kind, const double g[3])
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (!std::isfinite(tau) || !(tau > 0)) return fail(c, TFSPH_E_INVALID_ARG, "tau must be finite and > 0");
    double gg[3] = {0, 0, 0};
    if (g) {
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(g[k])) return fail(c, TFSPH_E_NONFINITE, "non-finite gravity");
            gg[k] = k < c->dim ? g[k] : 0.0;
        }
    }
    LaunchCtx L = lctx(c);
    const int64_t launches0 = c->launches;
    if (t_stop && c->D.n > 0) {
        if (mem_kind == TFSPH_MEM_HOST) {
            const size_t bytes = (size_t)c->D.n * c->tsize;
            if (c->precision == TFSPH_FP64) {
                const double *t = static_cast<const double *>(t_stop);
                for (int64_t j = 0; j < c->D.n; ++j)
                    if (!(t[j] > 0) || !std::isfinite(t[j])) return fail(c, TFSPH_E_NONFINITE, "t_stop must be finite and > 0");
            } else {
                const float *t = static_cast<const float *>(t_stop);
                for (int64_t j = 0; j < c->D.n; ++j)
                    if (!(t[j] > 0) || !std::isfinite(t[j])) return fail(c, TFSPH_E_NONFINITE, "t_stop must be finite and > 0");
            }
            TF_CUDA(c, cudaMemcpyAsync(c->staging, t_stop, bytes, cudaMemcpyHostToDevice, c->stream));
            TF_CUDA(c, launch_set_tstop(L, c->D, c->staging));
            c->launches += 1;
        } else if (mem_kind == TFSPH_MEM_DEVICE) {
            TF_CUDA(c, launch_set_tstop(L, c->D, t_stop));
            c->launches += 1;
        } else {
            return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
        }
    }
    cudaEvent_t *ev = nullptr;
    int rc = next_events(c, &ev);
    if (rc) return rc;
    if (ev) TF_CUDA(c, cudaEventRecord(ev[0], c->stream));
    rc = forward_quantities(c, ev);
    if (rc) return rc;
    StepArgs S;
    S.tau = tau;
    S.g[0] = gg[0];
    S.g[1] = gg[1];
    S.g[2] = gg[2];
    S.tstar_mode = c->p.tstar_mode;
    S.cell_acc = c->cell_acc;
    S.has_frozen = c->has_frozen ? 1 : 0;
    if (c->p.drag == TFSPH_DRAG_IDIC) {
        TF_CUDA(c, launch_cell_update(L, c->geo, c->phys, c->G, c->D, c->acc, S));
        c->launches += 1;
    } else {
        // ISPH needs the dust density (its interpolations divide by it); both
        // schemes then run the cross-phase sums and the update
        if (c->D.n > 0 && c->p.drag == TFSPH_DRAG_ISPH) {
            TF_CUDA(c, launch_density(L, c->geo, c->phys, c->D, c->rho_d, false, nullptr, nullptr));
            c->launches += 1;
        }
        TF_CUDA(c, launch_xdrag(L, c->geo, c->phys, c->G, c->D, c->rho_g, c->rho_d, c->acc, c->xb, S, c->p.drag));
        c->launches += 2 * ((c->G.n > 0 ? 1 : 0) + (c->D.n > 0 ? 1 : 0));
    }
    if (ev) {
        TF_CUDA(c, cudaEventRecord(ev[TFSPH_PROF_DRAG + 1], c->stream));
        c->prof_steps += 1;
        c->prof_launches += c->launches - launches0;
    }
    c->prepared = false;
    c->forced = false;
    c->nbl_valid = false;
    c->steps += 1;
    return TFSPH_OK;
}

int tfsph_profile(tfsph_ctx *c, int enable)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (enable) {
        TF_CUDA(c, cudaStreamSynchronize(c->stream));
        c->prof_used = 0;
        for (double &m : c->prof_ms) m = 0.0;
        c->prof_steps = 0;
        c->prof_launches = 0;
    }
    c->profiling = enable != 0;
    return TFSPH_OK;
}

int tfsph_profile_read(tfsph_ctx *c, double *ms, int64_t *steps, int64_t *launches)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    int rc = fold_profile(c);
    if (rc) return rc;
    if (ms)
        for (int k = 0; k < TFSPH_PROF_NPHASE; ++k) ms[k] = c->prof_ms[k];
    if (steps) *steps = c->prof_steps;
    if (launches) *launches = c->prof_launches;
    return TFSPH_OK;
}

int tfsph_step_adjoint(tfsph_ctx *c, double tau, const double g[3], void *lam_gx, void *lam_gv, void *lam_dx,
                       void *lam_du, void *lam_ts, int mem_kind)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (!std::isfinite(tau) || !(tau > 0)) return fail(c, TFSPH_E_INVALID_ARG, "tau must be finite and > 0");
    if (c->p.eos != TFSPH_EOS_ISOTHERMAL || c->p.av_alpha > 0 || c->p.av_beta > 0 || c->p.drag != TFSPH_DRAG_IDIC)
        return fail(c, TFSPH_E_INVALID_ARG,
                    "the adjoint covers the isothermal gas without artificial viscosity and the IDIC drag");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
    const int64_t ng = c->G.n, nd = c->D.n;
    if ((ng > 0 && (!lam_gx || !lam_gv)) || (nd > 0 && (!lam_dx || !lam_du || !lam_ts)))
        return fail(c, TFSPH_E_INVALID_ARG, "NULL adjoint array");
    double gg[3] = {0, 0, 0};
    if (g)
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(g[k])) return fail(c, TFSPH_E_NONFINITE, "non-finite gravity");
            gg[k] = k < c->dim ? g[k] : 0.0;
        }
    int rc;
    const size_t v4 = 4 * c->tsize, d = (size_t)c->dim;
    if (!c->adj_gx4) {
        if ((rc = dalloc(c, &c->adj_gx4, (size_t)ng * v4))) return rc;
        if ((rc = dalloc(c, &c->adj_gv4, (size_t)ng * v4))) return rc;
        if ((rc = dalloc(c, &c->adj_dx4, (size_t)nd * v4))) return rc;
        if ((rc = dalloc(c, &c->adj_du4, (size_t)nd * v4))) return rc;
        if ((rc = dalloc(c, &c->adj_lA, (size_t)ng * v4))) return rc;
        if ((rc = dalloc(c, &c->adj_out, (size_t)ng * v4))) return rc;
        if ((rc = dalloc(c, &c->adj_lrho, (size_t)ng * c->tsize))) return rc;
        if ((rc = dalloc(c, &c->adj_lts, (size_t)nd * c->tsize))) return rc;
    }
    // device views of the caller's arrays (component-major, id order)
    void *dgx = lam_gx, *dgv = lam_gv, *ddx = lam_dx, *ddu = lam_du, *dts = lam_ts;
    const size_t bg = d * (size_t)ng * c->tsize, bd = d * (size_t)nd * c->tsize, bt = (size_t)nd * c->tsize;
    if (mem_kind == TFSPH_MEM_HOST) {
        if (!c->adj_host && (rc = dalloc(c, &c->adj_host, 2 * bg + 2 * bd + bt))) return rc;
        char *base = static_cast<char *>(c->adj_host);
        dgx = base;
        dgv = base + bg;
        ddx = base + 2 * bg;
        ddu = base + 2 * bg + bd;
        dts = base + 2 * bg + 2 * bd;
        if (ng > 0) {
            TF_CUDA(c, cudaMemcpyAsync(dgx, lam_gx, bg, cudaMemcpyHostToDevice, c->stream));
            TF_CUDA(c, cudaMemcpyAsync(dgv, lam_gv, bg, cudaMemcpyHostToDevice, c->stream));
        }
        if (nd > 0) {
            TF_CUDA(c, cudaMemcpyAsync(ddx, lam_dx, bd, cudaMemcpyHostToDevice, c->stream));
            TF_CUDA(c, cudaMemcpyAsync(ddu, lam_du, bd, cudaMemcpyHostToDevice, c->stream));
            TF_CUDA(c, cudaMemcpyAsync(dts, lam_ts, bt, cudaMemcpyHostToDevice, c->stream));
        }
    }
    LaunchCtx L = lctx(c);
    // forward quantities of the step: binning, density, pressure acceleration
    if ((rc = forward_quantities(c))) return rc;
    // adjoint vectors into storage order
    TF_CUDA(c, launch_lam_gather_all(L, c->G, c->D, dgx, dgv, ddx, ddu, c->adj_gx4, c->adj_gv4, c->adj_dx4,
                                     c->adj_du4, c->adj_lts));
    StepArgs S;
    S.tau = tau;
    S.g[0] = gg[0];
    S.g[1] = gg[1];
    S.g[2] = gg[2];
    S.tstar_mode = c->p.tstar_mode;
    S.cell_acc = c->cell_acc;
    S.has_frozen = c->has_frozen ? 1 : 0;
    // update and cell drag -> lambda_A, lambda_v, lambda_u, lambda_t_stop
    TF_CUDA(c, launch_cell_adjoint(L, c->geo, c->phys, c->G, c->D, c->acc, S, c->adj_gx4, c->adj_gv4, c->adj_dx4,
                                   c->adj_du4, c->adj_lA, c->adj_lts));
    if (ng > 0) {
        // pressure force -> lambda_x (through d_ab) and lambda_q; q = cs^2/rho -> lambda_rho; density -> lambda_x
        TF_CUDA(c, launch_force_adjoint(L, c->geo, c->phys, c->G, c->adj_lA, c->adj_out));
        TF_CUDA(c, launch_lamq_to_lamrho(L, c->G, c->adj_out, c->rho_g, c->p.cs * c->p.cs, c->adj_lrho));
        TF_CUDA(c, launch_density_adjoint(L, c->geo, c->phys, c->G, c->adj_lrho, c->adj_out));
    }
    // lambda_x (+ the pair terms), lambda_v, lambda_u and lambda_t_stop back to id order
    TF_CUDA(c, launch_lam_scatter_all(L, c->G, c->D, c->adj_gx4, c->adj_out, c->adj_gv4, c->adj_du4, c->adj_lts, dgx,
                                      dgv, ddu, dts));
    if (mem_kind == TFSPH_MEM_HOST) {
        if (ng > 0) {
            TF_CUDA(c, cudaMemcpyAsync(lam_gx, dgx, bg, cudaMemcpyDeviceToHost, c->stream));
            TF_CUDA(c, cudaMemcpyAsync(lam_gv, dgv, bg, cudaMemcpyDeviceToHost, c->stream));
        }
        if (nd > 0) {
            TF_CUDA(c, cudaMemcpyAsync(lam_du, ddu, bd, cudaMemcpyDeviceToHost, c->stream));
            TF_CUDA(c, cudaMemcpyAsync(lam_ts, dts, bt, cudaMemcpyDeviceToHost, c->stream));
        }
        TF_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return TFSPH_OK;
}

// Snapshot blob: the header; for gas and dust in storage order (the order of
// the binning below) pos, vel (V4) and id; then the state's forward
// quantities: the cell starts of gas and dust (ncells + 1 each), the gas
// densities and the gas pressure accelerations (V4). Loading one leaves the
// context as a step would find it after its binning, density and force.
namespace {
struct SnapHeader {
    uint64_t magic;  // "TFSPHST2"
    int64_t n_gas, n_dust, steps;
    int32_t dim, precision;
    uint32_t ncells, reserved0;
    uint64_t reserved[3];
};
constexpr uint64_t kSnapMagic = 0x3254535048504654ull;

__global__ void k_check_snapshot(const SnapHeader *h, int64_t ng, int64_t nd, int dim, int precision,
                                 uint32_t ncells, int *err)
{
    if (h->magic != kSnapMagic || h->n_gas != ng || h->n_dust != nd || h->dim != dim || h->precision != precision ||
        h->ncells != ncells)
        atomicOr(err, kErrInternal);
}

// One region of the blob: a device array of the context and its size.
struct SnapPart {
    void *ptr;
    size_t bytes;
};

// One launch copies every part of a device snapshot (word by word: every
// part size and offset is a multiple of 4 bytes) and, when saving, writes the
// header, instead of one copy call per array.
constexpr int kCopyParts = 12;
constexpr int kHeaderWords = (int)(sizeof(SnapHeader) / 4);
static_assert(sizeof(SnapHeader) % 4 == 0, "snapshot header is copied in words");
struct CopyList {
    const uint32_t *src[kCopyParts];
    uint32_t *dst[kCopyParts];
    uint64_t words[kCopyParts];
    int n;
    uint32_t head[kHeaderWords];
    uint32_t *head_dst;  // NULL: no header to write
};

__global__ void __launch_bounds__(256) k_copy_words(CopyList L)
{
    if (L.head_dst && blockIdx.x == 0 && threadIdx.x < kHeaderWords) L.head_dst[threadIdx.x] = L.head[threadIdx.x];
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int s = 0; s < L.n; ++s) {
        const uint32_t *__restrict__ src = L.src[s];
        uint32_t *__restrict__ dst = L.dst[s];
        for (uint64_t i = t; i < L.words[s]; i += stride) dst[i] = src[i];
    }
}

std::vector<SnapPart> snap_parts(tfsph_ctx *c)
{
    const size_t v4 = 4 * c->tsize, nc = (size_t)c->ncells + 1;
    std::vector<SnapPart> parts;
    for (PhaseBufs *P : {&c->G, &c->D}) {
        const size_t n = (size_t)P->n;
        parts.push_back({P->pos[P->cur], n * v4});
        parts.push_back({P->vel[P->cur], n * v4});
        parts.push_back({P->id[P->cur], n * 4});
    }
    parts.push_back({c->G.start, nc * 4});
    parts.push_back({c->D.start, nc * 4});
    parts.push_back({c->rho_g, (size_t)c->G.n * c->tsize});
    parts.push_back({c->acc, (size_t)c->G.n * v4});
    return parts;
}
}  // namespace

int tfsph_state_bytes(const tfsph_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return TFSPH_E_INVALID_ARG;
    size_t total = sizeof(SnapHeader);
    for (const SnapPart &q : snap_parts(const_cast<tfsph_ctx *>(c))) total += q.bytes;
    *bytes = (int64_t)total;
    return TFSPH_OK;
}

int tfsph_save_state(tfsph_ctx *c, void *buf, int mem_kind)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (!buf) return fail(c, TFSPH_E_INVALID_ARG, "buf is NULL");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
    int rc = forward_quantities(c);
    if (rc) return rc;
    SnapHeader h{};
    h.magic = kSnapMagic;
    h.n_gas = c->G.n;
    h.n_dust = c->D.n;
    h.steps = c->steps;
    h.dim = c->dim;
    h.precision = c->precision;
    h.ncells = c->ncells;
    char *dst = static_cast<char *>(buf);
    if (mem_kind == TFSPH_MEM_DEVICE) {
        if (reinterpret_cast<uintptr_t>(buf) % 4 != 0) return fail(c, TFSPH_E_INVALID_ARG, "buf must be 4-byte aligned");
        CopyList L{};
        memcpy(L.head, &h, sizeof h);
        L.head_dst = reinterpret_cast<uint32_t *>(dst);
        dst += sizeof h;
        for (const SnapPart &q : snap_parts(c)) {
            if (q.bytes) {
                L.src[L.n] = static_cast<const uint32_t *>(q.ptr);
                L.dst[L.n] = reinterpret_cast<uint32_t *>(dst);
                L.words[L.n] = q.bytes / 4;
                ++L.n;
            }
            dst += q.bytes;
        }
        k_copy_words<<<4 * 152, 256, 0, c->stream>>>(L);
        TF_CUDA(c, cudaGetLastError());
        c->launches += 1;
        return TFSPH_OK;
    }
    memcpy(dst, &h, sizeof h);
    dst += sizeof h;
    for (const SnapPart &q : snap_parts(c)) {
        if (q.bytes) TF_CUDA(c, cudaMemcpyAsync(dst, q.ptr, q.bytes, cudaMemcpyDeviceToHost, c->stream));
        dst += q.bytes;
    }
    TF_CUDA(c, cudaStreamSynchronize(c->stream));  // complete on return
    return TFSPH_OK;
}

int tfsph_load_state(tfsph_ctx *c, const void *buf, int mem_kind)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (!buf) return fail(c, TFSPH_E_INVALID_ARG, "buf is NULL");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
    SnapHeader h{};
    const char *src = static_cast<const char *>(buf);
    if (mem_kind == TFSPH_MEM_DEVICE) {
        // checked on the device, without a host round trip; a mismatch is
        // reported by the next tfsph_sync (the copies below use this
        // context's sizes, so they stay in bounds either way)
        k_check_snapshot<<<1, 1, 0, c->stream>>>(reinterpret_cast<const SnapHeader *>(src), c->G.n, c->D.n, c->dim,
                                                 c->precision, c->ncells, c->d_err);
        TF_CUDA(c, cudaGetLastError());
        c->launches += 1;
        h.steps = -1;
    } else {
        memcpy(&h, src, sizeof h);
        if (h.magic != kSnapMagic || h.n_gas != c->G.n || h.n_dust != c->D.n || h.dim != c->dim ||
            h.precision != c->precision || h.ncells != c->ncells)
            return fail(c, TFSPH_E_INVALID_ARG, "snapshot does not belong to a context of this shape");
    }
    src += sizeof h;
    if (mem_kind == TFSPH_MEM_DEVICE) {
        if (reinterpret_cast<uintptr_t>(buf) % 4 != 0) return fail(c, TFSPH_E_INVALID_ARG, "buf must be 4-byte aligned");
        CopyList L{};
        for (const SnapPart &q : snap_parts(c)) {
            if (q.bytes) {
                L.src[L.n] = reinterpret_cast<const uint32_t *>(src);
                L.dst[L.n] = static_cast<uint32_t *>(q.ptr);
                L.words[L.n] = q.bytes / 4;
                ++L.n;
            }
            src += q.bytes;
        }
        k_copy_words<<<4 * 152, 256, 0, c->stream>>>(L);
        TF_CUDA(c, cudaGetLastError());
        c->launches += 1;
    } else {
        for (const SnapPart &q : snap_parts(c)) {
            if (q.bytes) TF_CUDA(c, cudaMemcpyAsync(q.ptr, src, q.bytes, cudaMemcpyHostToDevice, c->stream));
            src += q.bytes;
        }
    }
    if (mem_kind == TFSPH_MEM_HOST) TF_CUDA(c, cudaStreamSynchronize(c->stream));
    // the cell keys are rewritten by the step's update before the next binning;
    // the per-cell counters are cleared by that binning
    c->prepared = true;
    c->forced = true;
    c->nbl_valid = false;  // the neighbour list is not part of a snapshot
    c->counts_dirty = true;
    if (h.steps >= 0) c->steps = h.steps;
    return TFSPH_OK;
}

int tfsph_max_dt(tfsph_ctx *c, double cfl, double *tau_out)
{
    if (!c || !tau_out) return fail(c, TFSPH_E_INVALID_ARG, "NULL argument");
    if (!(cfl > 0) || !std::isfinite(cfl)) return fail(c, TFSPH_E_INVALID_ARG, "cfl must be finite and > 0");
    double vmax = c->p.cs;
    if (c->G.n > 0) {
        LaunchCtx L = lctx(c);
        TF_CUDA(c, launch_max_speed(L, c->phys, c->G, c->partials, c->npart, c->scalar));
        if (c->precision == TFSPH_FP64) {
            TF_CUDA(c, cudaMemcpyAsync(&vmax, c->scalar, 8, cudaMemcpyDeviceToHost, c->stream));
            TF_CUDA(c, cudaStreamSynchronize(c->stream));
        } else {
            float v = 0;
            TF_CUDA(c, cudaMemcpyAsync(&v, c->scalar, 4, cudaMemcpyDeviceToHost, c->stream));
            TF_CUDA(c, cudaStreamSynchronize(c->stream));
            vmax = v;
        }
    }
    if (!(vmax > 0)) return fail(c, TFSPH_E_INTERNAL, "no moving gas particle with a nonzero signal speed");
    *tau_out = cfl * c->p.h / vmax;
    return TFSPH_OK;
}

int tfsph_fields(tfsph_ctx *c, int field, void *out, int mem_kind, int order)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (order != TFSPH_ORDER_ORIGINAL && order != TFSPH_ORDER_CELL) return fail(c, TFSPH_E_INVALID_ARG, "bad order");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
    const PhaseBufs *P;
    int what, ncomp;
    const void *aux = nullptr;
    LaunchCtx L = lctx(c);
    int rc;
    switch (field) {
        case TFSPH_FIELD_POS_G: P = &c->G; what = 0; ncomp = c->dim; break;
        case TFSPH_FIELD_VEL_G: P = &c->G; what = 1; ncomp = c->dim; break;
        case TFSPH_FIELD_ENERGY_G: P = &c->G; what = 2; ncomp = 1; break;
        case TFSPH_FIELD_RHO_G:
            if ((rc = prepare(c))) return rc;
            P = &c->G; what = 3; ncomp = 1; aux = c->rho_g;
            break;
        case TFSPH_FIELD_POS_D: P = &c->D; what = 0; ncomp = c->dim; break;
        case TFSPH_FIELD_VEL_D: P = &c->D; what = 1; ncomp = c->dim; break;
        case TFSPH_FIELD_TSTOP_D: P = &c->D; what = 2; ncomp = 1; break;
        case TFSPH_FIELD_RHO_D:
            if ((rc = prepare(c))) return rc;
            TF_CUDA(c, launch_density(L, c->geo, c->phys, c->D, c->rho_d, false, nullptr, nullptr));
            P = &c->D; what = 3; ncomp = 1; aux = c->rho_d;
            break;
        default: return fail(c, TFSPH_E_INVALID_ARG, "unknown field");
    }
    if (P->n == 0) return TFSPH_OK;
    if (!out) return fail(c, TFSPH_E_INVALID_ARG, "out is NULL");
    const size_t bytes = (size_t)ncomp * (size_t)P->n * c->tsize;
    if (mem_kind == TFSPH_MEM_HOST && order == TFSPH_ORDER_CELL) {
        // a page-locked host buffer is written by the kernel directly when the
        // writes are in storage order; in id order they scatter over the host
        // link, so those go through the staging buffer and one bulk copy
        if (void *m = mapped_host(out)) {
            TF_CUDA(c, launch_unpack(L, *P, what, m, order, aux));
            TF_CUDA(c, cudaStreamSynchronize(c->stream));
            return TFSPH_OK;
        }
    }
    void *dst = mem_kind == TFSPH_MEM_DEVICE ? out : c->staging;
    if (mem_kind == TFSPH_MEM_HOST && bytes > c->staging_bytes) return fail(c, TFSPH_E_INTERNAL, "staging too small");
    TF_CUDA(c, launch_unpack(L, *P, what, dst, order, aux));
    return emit(c, dst, bytes, out, mem_kind);
}

int tfsph_debug(tfsph_ctx *c, int what, void *out, int mem_kind)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    if (!out) return fail(c, TFSPH_E_INVALID_ARG, "out is NULL");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return fail(c, TFSPH_E_INVALID_ARG, "bad mem_kind");
    LaunchCtx L = lctx(c);
    int rc;
    if (what == TFSPH_DEBUG_ACC_G) {
        // storage order of the last step is still current until the next binning
        if (c->G.n == 0) return TFSPH_OK;
        PhaseBufs Q = c->G;
        const size_t bytes = (size_t)c->dim * (size_t)c->G.n * c->tsize;
        void *dst = mem_kind == TFSPH_MEM_DEVICE ? out : c->staging;
        // reuse the unpack kernel: acc as "pos" of a phase view
        Q.pos[Q.cur] = c->acc;
        TF_CUDA(c, launch_unpack(L, Q, 0, dst, TFSPH_ORDER_ORIGINAL, nullptr));
        return emit(c, dst, bytes, out, mem_kind);
    }
    if ((rc = prepare(c))) return rc;
    const PhaseBufs &P = (what == TFSPH_DEBUG_KEYS_D || what == TFSPH_DEBUG_PERM_D || what == TFSPH_DEBUG_CSTART_D) ? c->D : c->G;
    void *dst = mem_kind == TFSPH_MEM_DEVICE ? out : c->staging;
    size_t bytes = 0;
    switch (what) {
        case TFSPH_DEBUG_KEYS_G:
        case TFSPH_DEBUG_KEYS_D:
            if (P.n == 0) return TFSPH_OK;
            TF_CUDA(c, launch_debug_keys(L, c->geo, P, static_cast<uint32_t *>(dst)));
            bytes = (size_t)P.n * 4;
            break;
        case TFSPH_DEBUG_PERM_G:
        case TFSPH_DEBUG_PERM_D:
            if (P.n == 0) return TFSPH_OK;
            k_mask_ids<<<(unsigned)((P.n + 255) / 256), 256, 0, c->stream>>>(P.id[P.cur], (int)P.n, static_cast<uint32_t *>(dst));
            TF_CUDA(c, cudaGetLastError());
            bytes = (size_t)P.n * 4;
            break;
        case TFSPH_DEBUG_CSTART_G:
        case TFSPH_DEBUG_CSTART_D:
            bytes = ((size_t)c->ncells + 1) * 4;
            if (mem_kind == TFSPH_MEM_DEVICE) TF_CUDA(c, cudaMemcpyAsync(out, P.start, bytes, cudaMemcpyDeviceToDevice, c->stream));
            else {
                TF_CUDA(c, cudaMemcpyAsync(out, P.start, bytes, cudaMemcpyDeviceToHost, c->stream));
                TF_CUDA(c, cudaStreamSynchronize(c->stream));
            }
            return TFSPH_OK;
        case TFSPH_DEBUG_NEIGH_COUNT:
        case TFSPH_DEBUG_NEIGH_FPRINT: {
            if (c->G.n == 0) return TFSPH_OK;
            const size_t n = (size_t)c->G.n;
            // counts and fingerprints into staging-sized temporaries
            void *cnt = nullptr, *fp = nullptr, *rho = nullptr;
            cudaError_t e = cudaMallocAsync(&cnt, n * 4, c->stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&fp, n * 8, c->stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&rho, n * c->tsize, c->stream);
            if (e == cudaSuccess)
                e = launch_density(L, c->geo, c->phys, c->G, rho, true, static_cast<int32_t *>(cnt),
                                   static_cast<uint64_t *>(fp));
            if (e == cudaSuccess) {
                const void *src = what == TFSPH_DEBUG_NEIGH_COUNT ? cnt : fp;
                const size_t b = n * (what == TFSPH_DEBUG_NEIGH_COUNT ? 4 : 8);
                e = cudaMemcpyAsync(out, src, b, mem_kind == TFSPH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
            }
            if (cnt) cudaFreeAsync(cnt, c->stream);
            if (fp) cudaFreeAsync(fp, c->stream);
            if (rho) cudaFreeAsync(rho, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "neighbour statistics");
            if (mem_kind == TFSPH_MEM_HOST) TF_CUDA(c, cudaStreamSynchronize(c->stream));
            return TFSPH_OK;
        }
        default: return fail(c, TFSPH_E_INVALID_ARG, "unknown debug export");
    }
    return emit(c, dst, bytes, out, mem_kind);
}

int tfsph_info(const tfsph_ctx *c, tfsph_info_t *out)
{
    if (!c || !out) return TFSPH_E_INVALID_ARG;
    out->n_gas = c->G.n;
    out->n_dust = c->D.n;
    for (int d = 0; d < 3; ++d) {
        out->n_cells[d] = c->ncell[d];
        out->reach[d] = c->reach[d];
    }
    out->n_cells_total = c->ncells;
    out->steps = c->steps;
    out->device_bytes = c->device_bytes;
    out->launches = c->launches;
    return TFSPH_OK;
}

int tfsph_sync(tfsph_ctx *c)
{
    if (!c) return fail(nullptr, TFSPH_E_INVALID_ARG, "ctx is NULL");
    TF_CUDA(c, cudaStreamSynchronize(c->stream));
    int err = 0;
    TF_CUDA(c, cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        TF_CUDA(c, cudaMemset(c->d_err, 0, sizeof(int)));
        if (err & kErrBadTstop) return fail(c, TFSPH_E_NONFINITE, "a t_stop value was <= 0 or not finite");
        return fail(c, TFSPH_E_INTERNAL, "device-side consistency check failed");
    }
    return TFSPH_OK;
}

}  // extern "C"
