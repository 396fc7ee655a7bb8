// api.cu -- host side of libvegasp: the C-ABI of include/vegasp.h.
//
// A context owns one "problem set" (one integral here; the batched entry
// points reuse the same machinery with many).  All state lives in one device
// arena per set, laid out member by member; kernels find it through a device
// array of descriptors.  Nothing per iteration crosses to the host: the
// iteration counter, the scale exponent, sum_h d_h and the allocation totals
// are device scalars, so an iterate+adapt pair can be captured once as a CUDA
// graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "host.h"

using namespace vp;

// ---------------------------------------------------------------------------
// errors and allocator
// ---------------------------------------------------------------------------
namespace vp {
thread_local std::string g_err = "no error";

vp_status fail(vp_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}
}  // namespace vp

static vp_alloc_fn g_alloc = nullptr;
static vp_free_fn g_free = nullptr;
static void *g_user = nullptr;

extern "C" vp_status vp_set_allocator(vp_alloc_fn alloc, vp_free_fn free_fn, void *user) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(VP_EINVAL, "vp_set_allocator: give both alloc and free, or neither");
    g_alloc = alloc;
    g_free = free_fn;
    g_user = user;
    return VP_OK;
}

extern "C" const char *vp_last_error(void) { return g_err.c_str(); }

namespace vp {
// Records a message for vp_last_error (used by entry points in other files).
const char *set_error_message(vp_status, const char *msg) {
    g_err = msg;
    return g_err.c_str();
}
}  // namespace vp

vp_status vp::dev_alloc(DevMem &m, size_t bytes, cudaStream_t s) {
    m.bytes = bytes;
    m.alloc = g_alloc;
    m.free_fn = g_free;
    m.user = g_user;
    if (bytes == 0) return VP_OK;
    if (m.alloc) {
        m.ptr = m.alloc(bytes, (void *)s, m.user);
        if (!m.ptr) return fail(VP_ENOMEM, "device allocation of %zu bytes failed", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(&m.ptr, bytes, s);
        if (e != cudaSuccess) {
            m.ptr = nullptr;
            cudaGetLastError();
            return fail(VP_ENOMEM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    return VP_OK;
}

void vp::dev_free(DevMem &m, cudaStream_t s) {
    if (!m.ptr) return;
    if (m.free_fn) m.free_fn(m.ptr, m.bytes, (void *)s, m.user);
    else cudaFreeAsync(m.ptr, s);
    m.ptr = nullptr;
}

// ---------------------------------------------------------------------------
// the problem set
// ---------------------------------------------------------------------------
struct Set {
    int device = 0;
    int n_sm = 0;
    std::vector<Member> m;
    std::vector<Desc> h_desc;
    std::vector<Group> groups;
    DevMem arena;
    Desc *d_desc = nullptr;
    uint32_t *d_tree_base = nullptr, *d_axis_base = nullptr;
    uint32_t n_tree_total = 0, n_axis_total = 0;
    int max_ng = 1;
    bool any_refine = false;
    cudaStream_t last = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the refinement (a8) runs on a side stream beside the estimate and the
    // reallocation (a6, a7): it reads only the histograms and the grid
    cudaStream_t side = nullptr;
    cudaEvent_t efork = nullptr, ejoin = nullptr;
    bool timed = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t iters = 0;  // iterations issued (host count)
    bool merge = false;  // one launch per (kind, precision): the largest bucket serves all
};

struct vp_ctx {
    Set set;
    // vp_step_read: two pinned slots {I_j, sigma_j^2}, filled on a side stream
    // from the iteration history (written once per iteration, so the copy may
    // trail the next step); step_ev marks a step's end, ev its copy's.
    // `pending`: slot ^ 1 holds a copy not yet returned.  t_off: the device's
    // iteration count minus set.iters (nonzero after an import).
    double *pin = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr}, step_ev[2] = {nullptr, nullptr};
    int slot = 0;
    bool pending = false;
    int64_t t_off = 0;
};

struct vp_batch {
    Set set;
};

int vp::bucket_of(int dim) {
    for (int b = 0; b < kNumBuckets; ++b)
        if (dim <= bucket_dim(b)) return b;
    return kNumBuckets - 1;
}

// Granlund-Montgomery constants for division by d (32-bit, round-up variant).
static void div_magic(uint32_t d, uint32_t *magic, int *shift) {
    if (d <= 1) {
        *magic = 0;
        *shift = 0;
        return;
    }
    int l = 0;
    while ((1ull << l) < d) ++l;  // ceil(log2 d)
    const unsigned __int128 num = ((unsigned __int128)1 << 32) * (((unsigned __int128)1 << l) - d);
    *magic = (uint32_t)(num / d + 1);
    *shift = l;
}

// floor((N_ev/4)^(1/D)) as the largest n >= 1 with 4 n^D <= N_ev.
// floor((N_ev/div)^(1/D)) as the largest n >= 1 with div n^D <= N_ev: div = 4
// is §3 Eq. (Nst_vegasp), div = 2 classic vegas's §3 Eq. (Nst).
static int64_t nstrat_exact(int dim, int64_t n_ev, int div) {
    auto fits = [&](int64_t n) {
        int64_t lim = n_ev / div, p = 1;
        for (int i = 0; i < dim; ++i) {
            if (p > lim / n) return false;
            p *= n;
        }
        return p <= lim;
    };
    if (n_ev < div) return 1;
    int64_t n = (int64_t)std::floor(std::pow((double)n_ev / (double)div, 1.0 / (double)dim));
    if (n < 1) n = 1;
    while (n > 1 && !fits(n)) --n;
    while (fits(n + 1)) ++n;
    return n;
}

// §3.2's mixed stratification: N_st + 1 strata on the first d axes, N_st on
// the others, N_st from Eq. (Nst_vegasp) and d the largest value with
// 4 (N_st + 1)^d N_st^(D - d) <= N_ev (integer arithmetic throughout).
static void nstrat_mixed_exact(int dim, int64_t n_ev, int div, std::vector<int64_t> &out) {
    const int64_t n = nstrat_exact(dim, n_ev, div), cap = n_ev / div;
    auto prod_fits = [&](int d) {  // (n + 1)^d n^(dim - d) <= cap
        int64_t p = 1;
        for (int mu = 0; mu < dim; ++mu) {
            const int64_t s = mu < d ? n + 1 : n;
            if (p > cap / s) return false;
            p *= s;
        }
        return true;
    };
    int d = 0;
    while (d < dim && prod_fits(d + 1)) ++d;
    out.assign(dim, n);
    for (int mu = 0; mu < d; ++mu) out[mu] = n + 1;
}

vp_status vp::validate(const vp_params *p, const vp_integrand *f, Member &mb) {
    if (!p || !f) return fail(VP_EINVAL, "NULL params or integrand");
    if (p->dim < 1 || p->dim > kMaxDim) return fail(VP_EINVAL, "dim %d outside 1..%d", p->dim, kMaxDim);
    if (p->n_g < 1 || p->n_g > kMaxNg) return fail(VP_EINVAL, "n_g %d outside 1..%d", p->n_g, kMaxNg);
    if (p->n_ev < 2) return fail(VP_EINVAL, "n_ev must be >= 2");
    if (!p->lo || !p->hi) return fail(VP_EINVAL, "NULL box");
    for (int i = 0; i < p->dim; ++i)
        if (!(std::isfinite(p->lo[i]) && std::isfinite(p->hi[i]) && p->lo[i] < p->hi[i]))
            return fail(VP_EINVAL, "box axis %d: need finite lo < hi", i);
    if (!(p->alpha >= 0.0 && std::isfinite(p->alpha))) return fail(VP_EINVAL, "alpha must be finite and >= 0");
    if (!(p->beta >= 0.0 && std::isfinite(p->beta))) return fail(VP_EINVAL, "beta must be finite and >= 0");
    if (p->precision != VP_FP64 && p->precision != VP_FP32) return fail(VP_EINVAL, "bad precision");
    if (p->n_st < 0) return fail(VP_EINVAL, "n_st must be >= 0");
    if (p->mixed != 0 && p->mixed != 1) return fail(VP_EINVAL, "mixed must be 0 or 1");
    if (p->n_st_axis)
        for (int i = 0; i < p->dim; ++i)
            if (p->n_st_axis[i] < 1) return fail(VP_EINVAL, "n_st_axis[%d] must be >= 1", i);
    if (p->d_weighted != 0 && p->d_weighted != 1) return fail(VP_EINVAL, "d_weighted must be 0 or 1");
    if (p->nst_div != 0 && p->nst_div != 2 && p->nst_div != 4)
        return fail(VP_EINVAL, "nst_div must be 0, 2 or 4");
    if (p->n_extra < 0 || p->n_extra > kMaxOut - 1)
        return fail(VP_EINVAL, "n_extra outside 0..%d", kMaxOut - 1);
    if (p->n_extra > 0) {
        if (!p->out_mono) return fail(VP_EINVAL, "NULL out_mono");
        if (p->precision != VP_FP64) return fail(VP_EINVAL, "several outputs: FP64 only");
        for (int i = 0; i < 2 * p->n_extra; ++i)
            if (p->out_mono[i] < -1 || p->out_mono[i] >= p->dim)
                return fail(VP_EINVAL, "out_mono[%d] outside -1..dim-1", i);
    }
    if (p->max_it < 0 || p->max_it > (1 << 24)) return fail(VP_EINVAL, "max_it outside 0..2^24");
    if (f->n_param < 1 || !f->param) return fail(VP_EINVAL, "empty integrand blob");
    const int D = p->dim;
    const double *q = f->param;
    const int n = f->n_param;
    switch (f->kind) {
        case VP_GAUSS:
        case VP_BALL:
        case VP_EXPNORM: {
            const double Kd = q[0];
            if (!(Kd >= 1 && Kd <= kMaxPeaks && Kd == std::floor(Kd)))
                return fail(VP_EINVAL, "peak count must be 1..%d", kMaxPeaks);
            const int K = (int)Kd;
            if (n != 1 + K * (2 + D)) return fail(VP_EINVAL, "blob needs %d doubles, got %d", 1 + K * (2 + D), n);
            break;
        }
        case VP_POSTERIOR: {
            if (n < 6) return fail(VP_EINVAL, "posterior blob too short");
            const double nd = q[0], Pd = q[1], Gd = q[2];
            if (!(nd >= 1 && nd <= kMaxPoints && nd == std::floor(nd)))
                return fail(VP_EINVAL, "posterior point count must be 1..%d", kMaxPoints);
            if (!(Pd >= 1 && Gd >= 1 && Pd == std::floor(Pd) && Gd == std::floor(Gd) && Pd + Gd == D))
                return fail(VP_EINVAL, "posterior needs P >= 1, G >= 1 and P + G = dim");
            const int np = (int)nd, P = (int)Pd;
            if (n != 6 + np + np * P) return fail(VP_EINVAL, "posterior blob needs %d doubles", 6 + np + np * P);
            if (!(q[3] > 0 && q[4] > 0)) return fail(VP_EINVAL, "posterior widths must be > 0");
            break;
        }
        default:
            return fail(VP_EINVAL, "unknown integrand kind %d", f->kind);
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(q[i])) return fail(VP_EINVAL, "non-finite integrand parameter %d", i);
    mb.p = *p;
    mb.kind = f->kind;
    mb.lo.assign(p->lo, p->lo + D);
    mb.hi.assign(p->hi, p->hi + D);
    mb.prm.assign(q, q + n);
    mb.p.lo = mb.lo.data();  // the caller's arrays may not outlive the call
    mb.p.hi = mb.hi.data();
    mb.p.n_st_axis = nullptr;  // (kept in nst_ax)
    mb.n_out = 1 + p->n_extra;
    mb.mono.assign(2, -1);
    if (p->n_extra > 0) mb.mono.insert(mb.mono.end(), p->out_mono, p->out_mono + 2 * p->n_extra);
    mb.p.out_mono = nullptr;  // (kept in mono)
    if (p->n_st_axis)
        mb.nst_ax.assign(p->n_st_axis, p->n_st_axis + D);
    else if (p->n_st > 0)
        mb.nst_ax.assign(D, p->n_st);
    else if (p->mixed)
        nstrat_mixed_exact(D, p->n_ev, p->nst_div ? p->nst_div : 4, mb.nst_ax);
    else
        mb.nst_ax.assign(D, nstrat_exact(D, p->n_ev, p->nst_div ? p->nst_div : 4));
    mb.n_st = *std::min_element(mb.nst_ax.begin(), mb.nst_ax.end());
    mb.uniform = *std::max_element(mb.nst_ax.begin(), mb.nst_ax.end()) == mb.n_st;
    // N_h = prod_mu s_mu <= 2^31
    uint64_t nh = 1;
    for (int i = 0; i < D; ++i) {
        nh *= (uint64_t)mb.nst_ax[i];
        if (nh > (1ull << 31)) return fail(VP_EINVAL, "the strata make more than 2^31 hypercubes");
    }
    mb.n_hc = nh;
    if (mb.n_out > 1 && nh > kMultiMaxHc)
        return fail(VP_EINVAL, "several outputs: at most %llu hypercubes",
                    (unsigned long long)kMultiMaxHc);
    const uint64_t calls = (uint64_t)((D + 3) / 4);
    const uint64_t max_nh = (uint64_t)p->n_ev + 2 * nh + 2;
    if (max_nh * calls >= (1ull << 32))
        return fail(VP_EINVAL, "(N_ev + 2 N_h) ceil(D/4) must stay below 2^32 (Philox counter word 0)");
    mb.n_tree = (uint32_t)((nh + kTreeBlock - 1) / kTreeBlock);
    mb.hist_cap = p->max_it > 0 ? p->max_it : 1024;
    mb.bucket = bucket_of(D);
    mb.exact = (D == bucket_dim(mb.bucket));
    // FP32 integrand constants
    const double L2E = 1.4426950408889634074;
    mb.prm32.clear();
    if (f->kind == VP_POSTERIOR) {
        const int np = (int)q[0], P = (int)q[1], G = (int)q[2];
        const double sy = q[3], pw = q[4], lref = q[5];
        const double s2pi = std::sqrt(2.0 * M_PI);
        mb.prm32.push_back((float)np);
        mb.prm32.push_back((float)P);
        mb.prm32.push_back((float)G);
        mb.prm32.push_back((float)(L2E / (2.0 * sy * sy)));
        mb.prm32.push_back((float)(L2E / (200.0 * sy * sy)));
        mb.prm32.push_back((float)std::log2(1.0 / (s2pi * sy)));
        mb.prm32.push_back((float)std::log2(1.0 / (s2pi * 10.0 * sy)));
        mb.prm32.push_back((float)(L2E / (2.0 * pw * pw)));
        mb.prm32.push_back((float)(lref * L2E));
        for (int i = 0; i < np; ++i) mb.prm32.push_back((float)q[6 + i]);
        for (int i = 0; i < np * P; ++i) mb.prm32.push_back((float)q[6 + np + i]);
    } else {
        // per peak {a, k, 0, 0, c[D], pad}: a multiple of 4 floats
        const int K = (int)q[0];
        const int D4 = (D + 3) & ~3;
        for (int k = 0; k < K; ++k) {
            const double *pk = q + 1 + k * (2 + D);
            mb.prm32.push_back((float)pk[0]);
            if (f->kind == VP_GAUSS) mb.prm32.push_back((float)(L2E / (pk[1] * pk[1])));
            else if (f->kind == VP_BALL) mb.prm32.push_back((float)(pk[1] * pk[1]));
            else mb.prm32.push_back((float)(pk[1] * L2E));
            mb.prm32.push_back(0.0f);
            mb.prm32.push_back(0.0f);
            for (int i = 0; i < D4; ++i) mb.prm32.push_back(i < D ? (float)pk[2 + i] : 0.0f);
        }
    }
    return VP_OK;
}

size_t vp::member_layout(Member &mb, size_t base) {
    const size_t D = mb.p.dim, G = mb.p.n_g, H = mb.n_hc, T = mb.n_tree, C = mb.hist_cap;
    const size_t M = mb.n_out > 1 ? mb.n_out : 0, MT = M * (M + 1) / 2;  // (App. B outputs)
    const size_t sz[B_COUNT] = {D * (G + 1) * 8, D * G * 8, mb.prm.size() * 8,
                                mb.prm32.size() * 4, H * 4, (H + 1) * 8, 2 * H * 8, 2 * H * 8,
                                H * 8, 2 * D * G * 8, 2 * D * G * 4, T * 15 * 8, T * kSub * 8, C * 8,
                                C * 8, sizeof(State), 2 * H * M * 8, 2 * H * MT * 8,
                                T * (M + MT) * 8, C * M * 8, C * MT * 8};
    for (int i = 0; i < B_COUNT; ++i) {
        mb.off_bytes[i] = base;
        base = align256(base + sz[i]);
    }
    return base;
}

// FP32 mirror {x_i, dx_i} of one axis.
static void make_tab(const double *e, int n_g, float2 *tab) {
    for (int i = 0; i < n_g; ++i) tab[i] = make_float2((float)e[i], (float)(e[i + 1] - e[i]));
}

// The precision every integral of a set takes (VP_FP32 or VP_FP64), or -1.
static int set_prec(const Set &s) {
    int p = s.h_desc.empty() ? -1 : s.h_desc[0].prec;
    for (const Desc &d : s.h_desc)
        if (d.prec != p) return -1;
    return p;
}

static vp_status plan_groups(Set &s) {
    // one launch group per (bucket, exactness, kind, precision); a merged set
    // (a batch) has one group per (kind, precision), served by the bucket of
    // its largest dimension
    int merged_bucket[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (const Member &mb : s.m)
        if (mb.n_out <= 1)  // (an integral with several outputs has a group of its own)
            merged_bucket[mb.kind][mb.p.precision] =
                std::max(merged_bucket[mb.kind][mb.p.precision], mb.bucket);
    for (uint32_t i = 0; i < s.m.size(); ++i) {
        const Member &mb = s.m[i];
        // several outputs (App. B): a group of its own, served by the FP64
        // one-integral kernel that sums them
        const bool solo = mb.n_out > 1;
        const int bucket = s.merge && !solo ? merged_bucket[mb.kind][mb.p.precision] : mb.bucket;
        // FP64 kernels are guarded; so is the task kernel's per-axis form
        // (several integrals with strata that differ between axes)
        bool exact = mb.exact && mb.p.precision == VP_FP32 && (mb.uniform || s.m.size() == 1);
        if (s.merge) {
            exact = mb.p.precision == VP_FP32;
            for (const Member &o : s.m)
                if (o.kind == mb.kind && o.p.precision == mb.p.precision && o.n_out <= 1 &&
                    (o.p.dim != bucket_dim(bucket) || !o.uniform))
                    exact = false;
        }
        Group *g = nullptr;
        for (auto &q : s.groups)
            if (!solo && !q.solo && q.bucket == bucket && q.exact == exact && q.kind == mb.kind &&
                q.prec == mb.p.precision)
                g = &q;
        if (!g) {
            s.groups.push_back(Group());
            g = &s.groups.back();
            g->bucket = bucket;
            g->exact = exact;
            g->kind = mb.kind;
            g->prec = mb.p.precision;
            g->solo = solo;
        }
        g->members.push_back(i);
    }
    std::vector<const Member *> mp;
    for (const Member &mb : s.m) mp.push_back(&mb);
    for (auto &g : s.groups) {
        vp_status st = group_config_many(mp, g, s.n_sm);
        if (st != VP_OK) return st;
        g.one = g.members.size() == 1;
        {
            // the one-integral kernel keeps FP32 peak constants in its
            // parameters: at most kParamPeaks peaks (else the task kernel)
            const Member &m0 = s.m[g.members[0]];
            if (g.prec == VP_FP32 && g.kind != VP_POSTERIOR && (int)m0.prm[0] > kParamPeaks)
                g.one = false;
        }
        // (strata that differ between axes, §3.2: the task kernel's per-axis
        // instantiation, g.uniform false, set by group_config_many; it has no
        // exact-dimension form, so such a group is exact only for the
        // one-integral kernel, and the task scheme is then not offered)
        g.mo = false;
        for (uint32_t i : g.members) g.mo = g.mo || s.m[i].n_out > 1;
        if (g.mo && !g.one)  // (not reached: such a member has a group of its own)
            return fail(VP_EINVAL, "several outputs: one integral per launch group");
        if (!g.uniform && g.exact && !g.one)
            return fail(VP_EINVAL, "strata that differ between axes: FP32 peaks at most %d",
                        kParamPeaks);
        if (!g.one) continue;
        {
            // a single FP32 peak at a dimension-exact bucket: the kernel's
            // single-peak form (see point32_p1)
            const Member &m0 = s.m[g.members[0]];
            g.p1 = g.prec == VP_FP32 && g.exact && g.kind != VP_POSTERIOR && !g.mo &&
                   (int)m0.prm[0] == 1;
        }
        // a single integral: the cluster kernel with its constants in parameters
        // (the autotuner may still choose the task kernel).  Its histograms:
        // the full shared layout (12 B per bin) when it fits one CTA per SM,
        // else the compact one (8 B; FP32 tiny terms go to global memory)
        {
            const size_t prm_bytes = (size_t)g.prm_words * 4;
            const size_t bins = (size_t)g.hist_words;
            if (prm_bytes + bins * 12 <= kOneSmemMax) {
                g.hist_one = kHistShared;
                g.smem_one = prm_bytes + bins * 12;
            } else if (g.prec == VP_FP32 && prm_bytes + bins * 8 <= kOneSmemMax) {
                g.hist_one = kHistCompact;
                g.smem_one = prm_bytes + bins * 8;
            } else {
                g.hist_one = kHistGlobal;
                g.smem_one = prm_bytes;
            }
        }
        cudaError_t e = g.prec == VP_FP64
                            ? sample_smem_config_f64(g.bucket, g.exact, g.kind, true, (int)std::max<size_t>(g.smem_one, 48 * 1024), g.mo)
                            : sample_smem_config_f32(g.bucket, g.exact, g.kind, true, (int)std::max<size_t>(g.smem_one, 48 * 1024), false, g.p1);
        if (e != cudaSuccess) return fail(VP_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
        g.occ_one = g.prec == VP_FP64
                        ? sample_occupancy_f64(g.bucket, g.exact, g.kind, true, g.threads, g.smem_one, g.mo)
                        : sample_occupancy_f32(g.bucket, g.exact, g.kind, true, g.threads, g.smem_one, false, g.p1);
        if (g.occ_one < 1) return fail(VP_ECUDA, "sampling kernel cannot be resident (smem %zu)", g.smem_one);
        g.blocks = s.n_sm * std::min(g.occ_one, 2);  // until the autotuner has measured
        if (g.hist_one) {
            // the largest cluster that keeps (nearly) every CTA slot busy
            int best = g.blocks;
            g.cs = 1;
            for (int cs : {2, 4, 8}) {  // (the kernel's reduction handles up to 8)
                const int ctas = g.prec == VP_FP64
                                     ? sample_cluster_ctas_f64(g.bucket, g.exact, g.kind, cs, g.blocks, g.threads, g.smem_one, g.mo)
                                     : sample_cluster_ctas_f32(g.bucket, g.exact, g.kind, cs, g.blocks, g.threads, g.smem_one, g.p1);
                if (ctas >= (int)(0.97 * g.blocks) && ctas >= cs) {
                    g.cs = cs;
                    best = ctas / cs * cs;
                }
            }
            g.blocks = best;
        }
        set_task(g, (double)s.m[g.members[0]].p.n_ev + 2.0 * (double)s.m[g.members[0]].n_hc);
        g.blocks_plan = g.blocks;
        g.cs_plan = g.cs;
        g.threads_plan = g.threads;
    }
    return VP_OK;
}

// Task-kernel launch shape of a group: shared-memory histograms when the
// largest member's fit (with the FP32 constants) in 112 KB, two CTAs per SM at
// most, tasks of ~1/8 of a CTA's share in whole warp chunks.
vp_status vp::group_config_many(const std::vector<const Member *> &m, Group &g, int n_sm) {
    double expect = 0.0;
    int max_bins = 0, max_words = 0;
    g.uniform = true;  // (else the per-axis instantiation of the task kernel)
    for (uint32_t i : g.members) g.uniform = g.uniform && m[i]->uniform;
    for (uint32_t i : g.members) {
        expect += (double)m[i]->p.n_ev + 2.0 * (double)m[i]->n_hc;
        max_bins = std::max(max_bins, m[i]->p.dim * m[i]->p.n_g);
        max_words = std::max(max_words, (int)m[i]->prm32.size());
    }
    // big integrals first: tasks of later members fill the tail
    std::stable_sort(g.members.begin(), g.members.end(), [&](uint32_t a, uint32_t b) {
        return m[a]->p.n_ev > m[b]->p.n_ev;
    });
    // per bin: an FP64 sum, or an FP32 sum and an FP32 tiny sum; a count
    const size_t hist_bytes = (size_t)max_bins * 12;
    g.threads = 256;
    g.r = 8;
    g.hist_words = max_bins;
    g.prm_words = g.prec == VP_FP64 ? 0 : ((max_words + 3) & ~3);
    const size_t prm_bytes = (size_t)g.prm_words * 4;
    g.hist_shared = (hist_bytes + prm_bytes <= 112 * 1024) ? 1 : 0;
    g.smem = prm_bytes + (g.hist_shared ? hist_bytes : 0);
    g.one = false;
    g.cs = 1;
    cudaError_t e = g.prec == VP_FP64
                        ? sample_smem_config_f64(g.bucket, g.exact, g.kind, false, (int)std::max<size_t>(g.smem, 48 * 1024), false, !g.uniform)
                        : sample_smem_config_f32(g.bucket, g.exact, g.kind, false, (int)std::max<size_t>(g.smem, 48 * 1024), !g.uniform);
    if (e != cudaSuccess) return fail(VP_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    g.occ_many = g.prec == VP_FP64
                     ? sample_occupancy_f64(g.bucket, g.exact, g.kind, false, g.threads, g.smem, false, !g.uniform)
                     : sample_occupancy_f32(g.bucket, g.exact, g.kind, false, g.threads, g.smem, !g.uniform);
    if (g.occ_many < 1) return fail(VP_ECUDA, "sampling kernel cannot be resident (smem %zu)", g.smem);
    g.blocks = n_sm * std::min(g.occ_many, 2);
    set_task(g, expect);
    return VP_OK;
}

// ---------------------------------------------------------------------------
// one member's descriptor and initial device state
// ---------------------------------------------------------------------------
// The FP32 path's constants of d_h = sigma_h^beta (§3 Eq. dh) with
// sigma_h = Omega sqrt(var): beta/2 as a sum of two floats, and
// beta log2(Omega) = -beta log2(N_h) as an integer plus a fraction in [0, 1).
void vp::damp_consts(Desc &d, double beta) {
    d.half_beta_hi = (float)(0.5 * beta);
    d.half_beta_lo = (float)(0.5 * beta - (double)d.half_beta_hi);
    const double c = -beta * std::log2((double)d.n_hc);
    const double ci = std::floor(c);
    d.lob_i = (int32_t)ci;
    d.lob_f = (float)(c - ci);
    if (d.lob_f >= 1.0f) {  // (the fraction rounded up to 1)
        d.lob_i += 1;
        d.lob_f = 0.0f;
    }
}

void vp::inv_table(std::vector<double> &inv) {
    inv.assign(kInvTabWords, 0.0);
    for (int k = 1; k < kInvTab; ++k) {
        double *e = inv.data() + 4 * k;
        e[0] = 1.0 / (double)k;  // IEEE division on the host
        if (k >= 2) e[1] = 1.0 / ((double)k * (double)(k - 1));  // (exact product)
        const double L = std::log2((double)k);
        float *l2 = (float *)(e + 2);
        l2[0] = (float)L;
        l2[1] = (float)(L - (double)l2[0]);
    }
}

void vp::fill_desc(const Member &mb, const double *d_inv, Desc &d) {
    const int D = mb.p.dim, G = mb.p.n_g;
    memset(&d, 0, sizeof d);
    d.dim = D;
    d.n_g = G;
    d.kind = mb.kind;
    d.prec = mb.p.precision;
    d.plus2 = mb.p.plus2 ? 1 : 0;
    d.n_peaks = (int)mb.prm[0];
    d.n_par = mb.kind == VP_POSTERIOR ? (int)mb.prm[1] : 0;
    d.hist_cap = mb.hist_cap;
    d.n_st = (uint32_t)mb.n_st;
    d.integral_id = mb.p.integral_id;
    d.key0 = (uint32_t)mb.p.seed;
    d.key1 = (uint32_t)(mb.p.seed >> 32);
    d.n_tree = mb.n_tree;
    d.n_ev = mb.p.n_ev;
    d.n_hc = mb.n_hc;
    d.omega = 1.0 / (double)mb.n_hc;
    d.omega2 = d.omega * d.omega;
    d.n_ev_d = (double)mb.p.n_ev;
    d.alpha = mb.p.alpha;
    d.beta = mb.p.beta;
    damp_consts(d, mb.p.beta);
    d.ng_over_nst = (float)((double)G / (double)mb.n_st);
    d.inv_ng = (float)(1.0 / (double)G);
    {
        int e = 0;
        const double m = std::frexp(std::pow((double)G, (double)D), &e);  // m in [0.5, 1)
        d.ngD_m = (float)(2.0 * m);
        d.ngD_e = e - 1;
    }
    div_magic((uint32_t)mb.n_st, &d.nst_magic, &d.nst_shift);
    d.uniform = mb.uniform ? 1u : 0u;
    d.n_out = mb.n_out;
    d.d_weighted = mb.p.d_weighted;
    for (int k = 0; k < 2 * kMaxOut; ++k) d.mono[k] = k < (int)mb.mono.size() ? mb.mono[k] : -1;
    if (mb.n_out > 1) {
        d.x1 = mbuf<double>(mb, B_X1);
        d.x2 = mbuf<double>(mb, B_X2);
        d.mpart = mbuf<double>(mb, B_MPART);
        d.hist_im = mbuf<double>(mb, B_HIM);
        d.hist_cm = mbuf<double>(mb, B_HCM);
    }
    d.n_st = (uint32_t)mb.nst_ax[0];
    for (int mu = 0; mu < kMaxDim; ++mu) {
        const uint32_t s = mu < D ? (uint32_t)mb.nst_ax[mu] : 1u;
        d.strata.n[mu] = s;
        div_magic(s, &d.strata.magic[mu], &d.strata.shift[mu]);
        d.strata.c32[mu] = (float)((double)G / (double)s);
        d.strata.nd[mu] = (double)s;
    }
    d.inv_tab = d_inv;
    d.edges = mbuf<double>(mb, B_EDGES);
    d.tab = mbuf<float2>(mb, B_TAB);
    d.prm = mbuf<double>(mb, B_PRM);
    d.prm32 = mbuf<float>(mb, B_PRM32);
    d.n_h = mbuf<uint32_t>(mb, B_NH);
    d.off = mbuf<uint64_t>(mb, B_OFF);
    d.s1 = mbuf<double>(mb, B_S1);
    d.s2 = mbuf<double>(mb, B_S2);
    d.dh = mbuf<double>(mb, B_DH);
    d.hsum = mbuf<double>(mb, B_HSUM);
    d.hcnt = mbuf<uint32_t>(mb, B_HCNT);
    d.part = mbuf<double>(mb, B_PART);
    d.bsum = mbuf<uint64_t>(mb, B_BSUM);
    d.hist_i = mbuf<double>(mb, B_HI);
    d.hist_var = mbuf<double>(mb, B_HV);
    d.st = mbuf<State>(mb, B_ST);
}

vp_status vp::upload_member_init(const Member &mb, const Desc &d, cudaStream_t stream) {
    const int D = mb.p.dim, G = mb.p.n_g;
    // uniform grid (§2.3: the first iteration uses a uniform grid)
    std::vector<double> edges((size_t)D * (G + 1));
    std::vector<float2> tab((size_t)D * G);
    double vol = 1.0;
    for (int mu = 0; mu < D; ++mu) {
        const double a = mb.lo[mu], b = mb.hi[mu];
        double *e = &edges[(size_t)mu * (G + 1)];
        for (int k = 0; k <= G; ++k) e[k] = a + (b - a) * (double)k / (double)G;
        e[0] = a;
        e[G] = b;
        make_tab(e, G, &tab[(size_t)mu * G]);
        vol *= (b - a);
    }
    State sti;
    memset(&sti, 0, sizeof sti);
    int e = std::ilogb(vol);
    sti.scale_exp = -(e > 120 ? 120 : (e < -120 ? -120 : e));
    std::vector<double> ones(mb.n_hc, 1.0);
    CU(cudaMemcpyAsync(d.edges, edges.data(), edges.size() * 8, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync(d.tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync((void *)d.prm, mb.prm.data(), mb.prm.size() * 8, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync((void *)d.prm32, mb.prm32.data(), mb.prm32.size() * 4, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync(d.dh, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync(d.st, &sti, sizeof sti, cudaMemcpyHostToDevice, stream));
    return VP_OK;
}

static vp_status set_create(Set &s, int n, const vp_params *ps, const vp_integrand *fs,
                            cudaStream_t stream) {
    if (n < 1 || !ps || !fs) return fail(VP_EINVAL, "need at least one integral");
    // host-side validation first: no CUDA call before the arguments are known good
    s.m.resize(n);
    for (int i = 0; i < n; ++i) {
        vp_status st = validate(&ps[i], &fs[i], s.m[i]);
        if (st != VP_OK) return st;
    }
    CU(cudaGetDevice(&s.device));
    CU(cudaDeviceGetAttribute(&s.n_sm, cudaDevAttrMultiProcessorCount, s.device));
    // arena layout: members, then descriptors and the set-level tables
    size_t base = 0;
    for (auto &mb : s.m) base = member_layout(mb, base);
    const size_t desc_off = base;
    base = align256(base + n * sizeof(Desc));
    const size_t tree_off = base;
    base = align256(base + (n + 1) * 4);
    const size_t axis_off = base;
    base = align256(base + (n + 1) * 4);
    const size_t inv_off = base;
    base = align256(base + kInvTabWords * sizeof(double));
    {
        vp_status pst = plan_groups(s);
        if (pst != VP_OK) return pst;
    }
    std::vector<size_t> gmem_off(s.groups.size() * 3);
    for (size_t g = 0; g < s.groups.size(); ++g) {
        gmem_off[3 * g] = base;
        base = align256(base + s.groups[g].members.size() * 4);
        gmem_off[3 * g + 1] = base;
        base = align256(base + (s.groups[g].members.size() + 1) * 8);
        gmem_off[3 * g + 2] = base;  // task queue head and exit counter, then the tail queues
        base = align256(base + 256 + (size_t)kTailQueues * kQueueStride * 4);
    }
    vp_status st = dev_alloc(s.arena, base, stream);
    if (st != VP_OK) return st;
    char *A = (char *)s.arena.ptr;
    CU(cudaMemsetAsync(A, 0, base, stream));
    s.d_desc = (Desc *)(A + desc_off);
    s.d_tree_base = (uint32_t *)(A + tree_off);
    s.d_axis_base = (uint32_t *)(A + axis_off);
    const double *d_inv = (const double *)(A + inv_off);
    {
        std::vector<double> inv;
        inv_table(inv);
        CU(cudaMemcpyAsync((void *)d_inv, inv.data(), kInvTabWords * sizeof(double),
                           cudaMemcpyHostToDevice, stream));
        CU(cudaStreamSynchronize(stream));
    }
    for (size_t g = 0; g < s.groups.size(); ++g) {
        s.groups[g].d_members = (uint32_t *)(A + gmem_off[3 * g]);
        s.groups[g].d_chunk_base = (uint64_t *)(A + gmem_off[3 * g + 1]);
        s.groups[g].d_head = (uint32_t *)(A + gmem_off[3 * g + 2]);
    }
    // host images of the initial state
    std::vector<uint32_t> tree_base(n + 1, 0), axis_base(n + 1, 0);
    s.h_desc.resize(n);
    for (int i = 0; i < n; ++i) {
        Member &mb = s.m[i];
        mb.base = A;
        fill_desc(mb, d_inv, s.h_desc[i]);
        vp_status ust = upload_member_init(mb, s.h_desc[i], stream);
        if (ust != VP_OK) return ust;
        tree_base[i + 1] = tree_base[i] + mb.n_tree;
        axis_base[i + 1] = axis_base[i] + mb.p.dim;
        s.max_ng = std::max(s.max_ng, mb.p.n_g);
        if (mb.p.alpha > 0.0 && mb.p.n_g > 1) s.any_refine = true;
    }
    CU(cudaStreamSynchronize(stream));
    s.n_tree_total = tree_base[n];
    s.n_axis_total = axis_base[n];
    for (auto &g : s.groups) {
        if (!g.one) continue;
        const Desc &d = s.h_desc[g.members[0]];
        const Member &mb = s.m[g.members[0]];
        SampleOne &a = g.args1;
        memset(&a, 0, sizeof a);
        Loop &L = a.L;  // the constants make_loop reads on the device
        L.dim = d.dim;
        L.n_g = d.n_g;
        L.K = d.n_peaks;
        L.nst_magic = d.nst_magic;
        L.nst_shift = d.nst_shift;
        L.n_st = d.n_st;
        L.calls = (uint32_t)((d.dim + 3) >> 2);
        L.iid = d.integral_id;
        L.dw = d.d_weighted;
        L.t = 0;
        uint32_t k0 = d.key0, k1 = d.key1;
        for (int r = 0; r < 10; ++r) {
            L.rk0[r] = k0;
            L.rk1[r] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        L.c32 = d.ng_over_nst;
        L.ngm1 = (float)(d.n_g - 1);
        L.ngD_m = d.ngD_m;
        L.ngD_e = d.ngD_e;
        L.nst = (double)d.n_st;
        L.ng = (double)d.n_g;
        L.tab = d.tab;
        L.edges = d.edges;
        a.S = d.strata;
        a.n_out = d.n_out;
        for (int k = 0; k < 2 * kMaxOut; ++k) a.mono[k] = d.mono[k];
        a.x1 = d.x1;
        a.x2 = d.x2;
        a.st = d.st;
        a.off = d.off;
        a.n_h = d.n_h;
        a.s1 = d.s1;
        a.s2 = d.s2;
        a.hsum = d.hsum;
        a.hcnt = d.hcnt;
        a.prm32 = d.prm32;
        a.prm = d.prm;
        a.n_hc = d.n_hc;
        a.head = g.d_head + kQueueStride;
        a.exit_count = g.d_head + 1;
        a.r = g.r;
        a.static16 = g.static16;
        a.hist_shared = g.hist_one;
        a.bins = d.dim * d.n_g;
        a.prm_words = g.prm_words;
        a.kp_peaks = 0;
        if (g.prec == VP_FP32 && g.kind != VP_POSTERIOR) {
            // {a, k, 0, 0, c[D], pad to 4} per peak -> {a, k, c[D]} at kParamStride
            const int K = (int)mb.prm[0], st = 4 + ((d.dim + 3) & ~3);
            for (int k = 0; k < K; ++k) {
                a.kp[k * kParamStride + 0] = mb.prm32[(size_t)k * st + 0];
                a.kp[k * kParamStride + 1] = mb.prm32[(size_t)k * st + 1];
                for (int mu = 0; mu < d.dim; ++mu)
                    a.kp[k * kParamStride + 2 + mu] = mb.prm32[(size_t)k * st + 4 + mu];
            }
            a.kp_peaks = K;
        }
    }
    CU(cudaMemcpyAsync(s.d_desc, s.h_desc.data(), n * sizeof(Desc), cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync(s.d_tree_base, tree_base.data(), (n + 1) * 4, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync(s.d_axis_base, axis_base.data(), (n + 1) * 4, cudaMemcpyHostToDevice, stream));
    for (auto &g : s.groups)
        CU(cudaMemcpyAsync(g.d_members, g.members.data(), g.members.size() * 4,
                           cudaMemcpyHostToDevice, stream));
    // first allocation: d_h = 1 -> max(2, floor(N_ev / N_h)) (the classic equal split)
    CU(launch_estimate(s.d_desc, s.d_tree_base, n, s.n_tree_total, 2, stream));
    CU(launch_alloc(s.d_desc, s.d_tree_base, n, s.n_tree_total, stream, 1));
    CU(cudaEventCreate(&s.ev0));
    CU(cudaEventCreate(&s.ev1));
    CU(cudaEventCreateWithFlags(&s.efork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&s.ejoin, cudaEventDisableTiming));
    CU(cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking));
    CU(cudaStreamSynchronize(stream));
    s.last = stream;
    return VP_OK;
}

static void set_destroy(Set &s) {
    if (!s.arena.ptr && !s.ev0) return;  // nothing was created on the device
    if (s.gexec) cudaGraphExecDestroy(s.gexec);
    if (s.graph) cudaGraphDestroy(s.graph);
    if (s.ev0) cudaEventDestroy(s.ev0);
    if (s.ev1) cudaEventDestroy(s.ev1);
    if (s.side) {
        cudaStreamSynchronize(s.side);
        cudaStreamDestroy(s.side);
    }
    if (s.efork) cudaEventDestroy(s.efork);
    if (s.ejoin) cudaEventDestroy(s.ejoin);
    cudaStreamSynchronize(s.last);
    dev_free(s.arena, s.last);
    cudaStreamSynchronize(s.last);
}

vp_status vp::launch_group(const Desc *d_desc, Group &g, cudaStream_t stream) {
    cudaError_t e;
    if (g.one) {
        e = g.prec == VP_FP64
                ? launch_sample_one_f64(g.bucket, g.exact, g.kind, g.blocks, g.threads_one, g.smem_one, g.cs, stream, g.args1)
                : launch_sample_one_f32(g.bucket, g.exact, g.kind, g.blocks, g.threads_one, g.smem_one, g.cs, stream, g.args1);
    } else {
        SampleArgs a;
        a.desc = d_desc;
        a.members = g.d_members;
        a.chunk_base = g.d_chunk_base;
        a.head = g.d_head;
        a.exit_count = g.d_head + 1;
        a.n_group = (int)g.members.size();
        a.r = g.r;
        a.task = g.task;
        a.hist_shared = g.hist_shared;
        a.hist_words = g.hist_words;
        a.prm_words = g.prm_words;
        e = g.prec == VP_FP64
                ? launch_sample_f64(g.bucket, g.exact, g.kind, g.blocks, g.threads, g.smem, stream, a, !g.uniform)
                : launch_sample_f32(g.bucket, g.exact, g.kind, g.blocks, g.threads, g.smem, stream, a, !g.uniform);
    }
    if (e != cudaSuccess) return fail(VP_ECUDA, "sampling launch: %s", cudaGetErrorString(e));
    return VP_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: time candidate launch shapes of the sampling kernel on the live
// state (the accumulators of the coming iteration are cleared afterwards, so
// the tuning samples leave no trace) and keep the fastest.  Candidates: the
// one-integral kernel (static balanced split) with 1..3 CTAs per SM and
// clusters of 1, 2, 4 or 8 CTAs, and the task kernel (dynamic work stealing)
// with 1..3 CTAs per SM and runs of 4 or 8 samples per thread.
// ---------------------------------------------------------------------------
struct Cand {
    bool one;
    int blocks, cs, r, threads, static16;
};

static vp_status time_group(Set &s, Group &g, cudaStream_t stream, float *best_ms) {
    float t[7];
    for (int rep = 0; rep < 7; ++rep) {
        if (!g.one)
            CU(launch_chunks(s.d_desc, g.d_members, (int)g.members.size(), g.d_chunk_base, g.d_head,
                             g.task, stream));
        CU(cudaEventRecord(s.ev0, stream));
        vp_status st = launch_group(s.d_desc, g, stream);
        if (st != VP_OK) return st;
        CU(cudaEventRecord(s.ev1, stream));
        CU(cudaEventSynchronize(s.ev1));
        CU(cudaEventElapsedTime(&t[rep], s.ev0, s.ev1));
    }
    std::sort(t + 1, t + 7);  // the first launch warms up; the median of the rest
    *best_ms = 0.5f * (t[3] + t[4]);
    return VP_OK;
}

// Tuning results are kept for the process, keyed by what decides the launch
// shape: kernel (precision, bucket, exactness, kind), histogram size, constants,
// number of integrals and the order of magnitude of their samples.
struct TuneKey {
    int prec, bucket, exact, kind, hist_shared, bins, prm_words, members, dev;
    int log2_samples;
    bool operator==(const TuneKey &o) const { return memcmp(this, &o, sizeof *this) == 0; }
};
struct TuneVal {
    bool one;
    int blocks, cs, r, threads, static16;
    bool final;  // measured on an adapted state
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

static TuneKey tune_key(const Set &s, const Group &g, double expect) {
    TuneKey k;
    memset(&k, 0, sizeof k);
    k.prec = g.prec;
    k.bucket = g.bucket;
    k.exact = g.exact;
    k.kind = g.kind;
    k.hist_shared = g.hist_shared * 4 + g.hist_one;
    k.bins = g.hist_words;
    k.prm_words = g.prm_words;
    k.members = (int)g.members.size();
    k.dev = s.device;
    k.log2_samples = (int)std::floor(std::log2(std::max(1.0, expect)));
    return k;
}

void vp::set_task(Group &g, double expect) {
    const uint32_t wchunk = 32u * (uint32_t)g.r;
    const double per = expect / ((double)g.blocks * 8.0);
    g.task = (uint32_t)std::min(1.0e9, std::max((double)(8 * wchunk), per));
    g.task = (g.task + wchunk - 1) / wchunk * wchunk;
}

// Launches of fewer samples than this keep the planned shape untuned.
constexpr double kTuneMinSamples = 262144.0;
// Launches of at least this many samples also try the dynamic tail.
constexpr double kTailMinSamples = 16777216.0;

static bool tune_due(const Set &s, const Group &g) {
    return !g.tuned || (!g.tuned_final && s.iters >= (uint64_t)kRetuneIt);
}

static vp_status tune(Set &s, cudaStream_t stream) {
    bool pending = false;
    for (auto &g : s.groups) pending |= tune_due(s, g);
    if (!pending) return VP_OK;
    CU(cudaStreamSynchronize(s.last));
    CU(cudaStreamSynchronize(stream));
    for (auto &g : s.groups) {
        if (!tune_due(s, g)) continue;
        const bool adapted = s.iters >= (uint64_t)kRetuneIt;
        {
            double expect0 = 0.0;
            for (uint32_t i : g.members) expect0 += (double)s.m[i].p.n_ev + 2.0 * (double)s.m[i].n_hc;
            const TuneKey key = tune_key(s, g, expect0);
            std::lock_guard<std::mutex> lock(g_tune_mu);
            bool hit = false;
            for (auto &kv : g_tune_cache)
                if (kv.first == key && (kv.second.final || !adapted)) {
                    g.one = kv.second.one;
                    g.blocks = kv.second.blocks;
                    g.cs = kv.second.cs;
                    g.r = kv.second.r;
                    g.threads_one = kv.second.threads;
                    g.static16 = kv.second.static16;
                    g.args1.r = g.r;
                    g.args1.static16 = g.static16;
                    set_task(g, expect0);
                    g.tuned = true;
                    g.tuned_final = kv.second.final;
                    hit = true;
                    break;
                }
            if (hit) continue;
        }
        std::vector<Cand> cands;
        const bool can_one = g.members.size() == 1;
        double expect = 0.0;
        for (uint32_t i : g.members) expect += (double)s.m[i].p.n_ev + 2.0 * (double)s.m[i].n_hc;
        if (expect < kTuneMinSamples) {  // a small launch: measuring costs more than it saves
            g.tuned = true;
            g.tuned_final = true;
            continue;
        }
        if (can_one && g.one) {
            // CTAs of 256 threads (1..3 per SM), or one larger CTA per SM
            const int max_threads = one_max_threads(bucket_dim(g.bucket), g.prec == VP_FP64, g.p1);
            for (int threads : {256, 512, 768, 1024}) {
                if (threads > max_threads) continue;
                const int occ = g.prec == VP_FP64
                                    ? sample_occupancy_f64(g.bucket, g.exact, g.kind, true, threads, g.smem_one, g.mo)
                                    : sample_occupancy_f32(g.bucket, g.exact, g.kind, true, threads, g.smem_one, false, g.p1);
                for (int k = 1; k <= std::min(threads == 256 ? 3 : 1, occ); ++k) {
                    const int blocks = k * s.n_sm;
                    for (int cs : {1, 2, 4, 8}) {
                        if (cs > 1 && !g.hist_one) continue;
                        int ctas = blocks;
                        if (cs > 1) {
                            ctas = g.prec == VP_FP64
                                       ? sample_cluster_ctas_f64(g.bucket, g.exact, g.kind, cs, blocks, threads, g.smem_one, g.mo)
                                       : sample_cluster_ctas_f32(g.bucket, g.exact, g.kind, cs, blocks, threads, g.smem_one, g.p1);
                            ctas = std::min(ctas, blocks) / cs * cs;
                            if (ctas < (int)(0.9 * blocks)) continue;
                        }
                        // (the dynamic tail, scheme 2, is timed below for large
                        // launches only, on the best static shape)
                        cands.push_back({true, ctas, cs, g.r, threads, kStaticShare});
                    }
                }
            }
        }
        if ((g.uniform || !g.exact) && !g.mo)
            for (int k = 1; k <= std::min(3, g.occ_many); ++k)
                for (int r : {4, 8}) cands.push_back({false, k * s.n_sm, 1, r, 256, 16});
        if (cands.size() <= 1) {
            g.tuned = true;
            g.tuned_final = true;
            continue;
        }
        const Cand keep = {g.one, g.blocks, g.cs, g.r, g.threads_one, g.static16};
        Cand best = keep;
        float best_ms = 1e30f;
        for (const Cand &c : cands) {
            g.one = c.one;
            g.blocks = c.blocks;
            g.cs = c.cs;
            g.r = c.r;
            g.threads_one = c.threads;
            g.static16 = c.static16;
            g.args1.r = c.r;
            g.args1.static16 = c.static16;
            set_task(g, expect);
            float ms = 0.f;
            vp_status st = time_group(s, g, stream, &ms);
            if (st != VP_OK) return st;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        if (best.one && expect >= kTailMinSamples) {
            // the best static shape with a dynamic tail (scheme 2): measured, the
            // SMs' differing speeds leave an even split waiting on the slowest
            // at large launches (the eight-D four peaks at N_ev = 1e8: 3.54 ->
            // 2.96 ms), while at small ones the queue costs more than it evens
            Cand twin = best;
            twin.static16 = kTailShare;
            g.one = twin.one;
            g.blocks = twin.blocks;
            g.cs = twin.cs;
            g.r = twin.r;
            g.threads_one = twin.threads;
            g.static16 = twin.static16;
            g.args1.r = twin.r;
            g.args1.static16 = twin.static16;
            set_task(g, expect);
            float ms = 0.f;
            vp_status st = time_group(s, g, stream, &ms);
            if (st != VP_OK) return st;
            if (ms < best_ms) {
                best_ms = ms;
                best = twin;
            }
        }
        g.one = best.one;
        g.blocks = best.blocks;
        g.cs = best.cs;
        g.r = best.r;
        g.threads_one = best.threads;
        g.static16 = best.static16;
        g.args1.r = best.r;
        g.args1.static16 = best.static16;
        set_task(g, expect);
        g.tuned = true;
        g.tuned_final = adapted;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            const TuneKey key = tune_key(s, g, expect);
            const TuneVal val = {g.one, g.blocks, g.cs, g.r, g.threads_one, g.static16, adapted};
            bool found = false;
            for (auto &kv : g_tune_cache)
                if (kv.first == key) {
                    if (adapted || !kv.second.final) kv.second = val;
                    found = true;
                }
            if (!found) g_tune_cache.push_back({key, val});
        }
        // clear what the tuning launches accumulated (buffer t & 1 of each member)
        for (uint32_t i : g.members) {
            const Desc &d = s.h_desc[i];
            State st;
            CU(cudaMemcpy(&st, d.st, sizeof st, cudaMemcpyDeviceToHost));
            const size_t par = st.t & 1u, bins = (size_t)d.dim * d.n_g;
            CU(cudaMemsetAsync(d.s1 + par * d.n_hc, 0, d.n_hc * 8, stream));
            CU(cudaMemsetAsync(d.s2 + par * d.n_hc, 0, d.n_hc * 8, stream));
            CU(cudaMemsetAsync(d.hsum + par * bins, 0, bins * 8, stream));
            CU(cudaMemsetAsync(d.hcnt + par * bins, 0, bins * 4, stream));
            if (d.n_out > 1) {
                const size_t M = (size_t)d.n_out, MT = M * (M + 1) / 2;
                CU(cudaMemsetAsync(d.x1 + par * d.n_hc * M, 0, d.n_hc * M * 8, stream));
                CU(cudaMemsetAsync(d.x2 + par * d.n_hc * MT, 0, d.n_hc * MT * 8, stream));
            }
        }
        CU(cudaStreamSynchronize(stream));
    }
    return VP_OK;
}

// Forks the refinement onto the side stream after what `stream` holds so far;
// join_refine makes `stream` wait for it.  (Inside a capture both become graph
// edges.)
static vp_status fork_refine(Set &s, cudaStream_t stream) {
    const int n = (int)s.m.size();
    CU(cudaEventRecord(s.efork, stream));
    CU(cudaStreamWaitEvent(s.side, s.efork, 0));
    CU(launch_refine(s.d_desc, s.d_axis_base, n, s.n_axis_total, s.max_ng, s.side));
    CU(cudaEventRecord(s.ejoin, s.side));
    return VP_OK;
}
static vp_status join_refine(Set &s, cudaStream_t stream) {
    CU(cudaStreamWaitEvent(stream, s.ejoin, 0));
    return VP_OK;
}

static vp_status set_iterate(Set &s, cudaStream_t stream, bool refine_too = false) {
    NvtxRange nv("vp.iterate");
    const int n = (int)s.m.size();
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusActive) {
        vp_status st = tune(s, stream);
        if (st != VP_OK) return st;
    }
    for (size_t gi = 0; gi < s.groups.size(); ++gi) {
        Group &g = s.groups[gi];
        if (!g.one)  // the task prefix (the one-integral kernel needs none)
            CU(launch_chunks(s.d_desc, g.d_members, (int)g.members.size(), g.d_chunk_base,
                             g.d_head, g.task, stream));
    }
    // the sampling launch is timed by events outside the step graph only: as
    // record nodes inside it they would add several microseconds to every step
    const bool timed = cap != cudaStreamCaptureStatusActive;
    if (timed) CU(cudaEventRecord(s.ev0, stream));
    for (size_t gi = 0; gi < s.groups.size(); ++gi) {
        vp_status st = launch_group(s.d_desc, s.groups[gi], stream);
        if (st != VP_OK) return st;
    }
    if (timed) {
        CU(cudaEventRecord(s.ev1, stream));
        s.timed = true;
    }
    if (cap != cudaStreamCaptureStatusActive) ++s.iters;
    for (int i = 0; i < n; ++i)
        if (s.m[i].n_out > 1)  // several outputs (App. B), before the counter advances
            CU(launch_estimate_multi(s.d_desc + i, s.m[i].n_tree, stream));
    if (refine_too && s.any_refine) {  // the step graph: a8 beside a6 and a7
        vp_status st = fork_refine(s, stream);
        if (st != VP_OK) return st;
    }
    CU(launch_estimate(s.d_desc, s.d_tree_base, n, s.n_tree_total, 0, stream, set_prec(s)));
    s.last = stream;
    return VP_OK;
}

static vp_status set_adapt(Set &s, cudaStream_t stream, bool refine_forked = false) {
    NvtxRange nv("vp.adapt");
    const int n = (int)s.m.size();
    if (s.any_refine && !refine_forked) {
        vp_status st = fork_refine(s, stream);
        if (st != VP_OK) return st;
    }
    CU(launch_alloc(s.d_desc, s.d_tree_base, n, s.n_tree_total, stream, 0));
    if (s.any_refine) {
        vp_status st = join_refine(s, stream);
        if (st != VP_OK) return st;
    }
    s.last = stream;
    return VP_OK;
}

static vp_status set_step(Set &s, cudaStream_t stream) {
    NvtxRange nv("vp.step");
    bool due = false;
    for (auto &g : s.groups) due |= tune_due(s, g);
    if (due && s.gexec) {  // a new launch shape: capture the step again
        CU(cudaStreamSynchronize(s.last));
        cudaGraphExecDestroy(s.gexec);
        cudaGraphDestroy(s.graph);
        s.gexec = nullptr;
        s.graph = nullptr;
    }
    if (!s.gexec) {
        vp_status tst = tune(s, stream);  // before the capture: tuning synchronises
        if (tst != VP_OK) return tst;
        // capture on a private stream so that the caller's stream may be the
        // legacy default stream (which cannot be captured)
        cudaStream_t cap;
        CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        CU(cudaStreamSynchronize(stream));
        CU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        vp_status st = set_iterate(s, cap, true);
        if (st == VP_OK) st = set_adapt(s, cap, true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (st != VP_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(VP_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        s.graph = g;
        CU(cudaGraphInstantiate(&s.gexec, s.graph, 0));
    }
    CU(cudaGraphLaunch(s.gexec, stream));
    ++s.iters;
    s.last = stream;
    return VP_OK;
}

// §2.5 combination of iterations j >= discard.
void vp::combine(const double *I, const double *V, int n, int discard, vp_result_t *r) {
    int first = discard < 0 ? 0 : discard;
    r->n_it = n > first ? n - first : 0;
    r->dof = r->n_it > 0 ? r->n_it - 1 : 0;
    r->mean = NAN;
    r->sdev = NAN;
    r->chi2 = NAN;
    if (r->n_it == 0) return;
    int zero = 0;
    double zsum = 0.0;
    for (int j = first; j < n; ++j)
        if (!(V[j] > 0.0)) {
            ++zero;
            zsum += I[j];
        }
    if (zero) {  // reading: zero-variance iterations are exact
        r->mean = zsum / zero;
        r->sdev = 0.0;
        r->chi2 = 0.0;
        return;
    }
    double sw = 0.0, swi = 0.0;
    for (int j = first; j < n; ++j) {
        sw += 1.0 / V[j];
        swi += I[j] / V[j];
    }
    r->mean = swi / sw;
    r->sdev = 1.0 / std::sqrt(sw);
    double c = 0.0;
    for (int j = first; j < n; ++j) c += (I[j] - r->mean) * (I[j] - r->mean) / V[j];
    r->chi2 = c;
}

// Eigen-decomposition of a symmetric M x M matrix (cyclic Jacobi rotations,
// Golub & Van Loan, "Matrix Computations", Sec. 8.5): A = U diag(w) U^T.
static void sym_eigen(int M, std::vector<double> A, std::vector<double> &w,
                      std::vector<double> &U) {
    U.assign((size_t)M * M, 0.0);
    for (int i = 0; i < M; ++i) U[(size_t)i * M + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, all = 0.0;
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                all += A[(size_t)i * M + j] * A[(size_t)i * M + j];
                if (i != j) off += A[(size_t)i * M + j] * A[(size_t)i * M + j];
            }
        if (off <= 1e-32 * all || off == 0.0) break;
        for (int p = 0; p < M - 1; ++p)
            for (int q = p + 1; q < M; ++q) {
                const double apq = A[(size_t)p * M + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * M + p], aqq = A[(size_t)q * M + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double tq = (theta >= 0.0 ? 1.0 : -1.0) /
                                  (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(tq * tq + 1.0), sn = tq * c;
                for (int k = 0; k < M; ++k) {  // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * M + p], akq = A[(size_t)k * M + q];
                    A[(size_t)k * M + p] = c * akp - sn * akq;
                    A[(size_t)k * M + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < M; ++k) {  // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * M + k], aqk = A[(size_t)q * M + k];
                    A[(size_t)p * M + k] = c * apk - sn * aqk;
                    A[(size_t)q * M + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < M; ++k) {  // U <- U J
                    const double ukp = U[(size_t)k * M + p], ukq = U[(size_t)k * M + q];
                    U[(size_t)k * M + p] = c * ukp - sn * ukq;
                    U[(size_t)k * M + q] = sn * ukp + c * ukq;
                }
            }
    }
    w.resize(M);
    for (int i = 0; i < M; ++i) w[i] = A[(size_t)i * M + i];
}

// Pseudo-inverse of a symmetric matrix: eigenvalues at or below `cut` times
// the largest magnitude are dropped.  Returns false if all are.
static bool sym_pinv(int M, const double *A, double cut, std::vector<double> &out) {
    std::vector<double> S((size_t)M * M), w, U;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j)
            S[(size_t)i * M + j] = 0.5 * (A[(size_t)i * M + j] + A[(size_t)j * M + i]);
    sym_eigen(M, S, w, U);
    double top = 0.0;
    for (double x : w) top = std::max(top, std::fabs(x));
    out.assign((size_t)M * M, 0.0);
    bool any = false;
    for (int e = 0; e < M; ++e) {
        if (!(top > 0.0 && w[e] > cut * top)) continue;
        any = true;
        const double inv = 1.0 / w[e];
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j)
                out[(size_t)i * M + j] += U[(size_t)i * M + e] * inv * U[(size_t)j * M + e];
    }
    return any;
}

// App. B's several integrals over iterations j >= discard: the several-variable
// form of §2.5's weighted average (generalised least squares; the paper
// states the one-variable form only).
int vp::combine_multi(const double *I, const double *C, int n, int M, int discard, double *mean,
                      double *cov, double *chi2) {
    const int first = discard < 0 ? 0 : discard;
    const int n_it = n > first ? n - first : 0;
    for (int k = 0; k < M; ++k) mean[k] = NAN;
    for (int q = 0; q < M * M; ++q) cov[q] = NAN;
    *chi2 = NAN;
    if (n_it == 0) return 0;
    const double cut = 1e-12;
    std::vector<std::vector<double>> W(n);
    std::vector<double> Ws((size_t)M * M, 0.0), rhs(M, 0.0);
    bool any = false;
    for (int j = first; j < n; ++j) {
        any |= sym_pinv(M, C + (size_t)j * M * M, cut, W[j]);
        for (int q = 0; q < M * M; ++q) Ws[q] += W[j][q];
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) rhs[a] += W[j][(size_t)a * M + b] * I[(size_t)j * M + b];
    }
    if (!any) {  // zero covariances: the plain mean
        for (int k = 0; k < M; ++k) {
            double s = 0.0;
            for (int j = first; j < n; ++j) s += I[(size_t)j * M + k];
            mean[k] = s / n_it;
        }
        for (int q = 0; q < M * M; ++q) cov[q] = 0.0;
        *chi2 = 0.0;
        return n_it;
    }
    std::vector<double> P;
    sym_pinv(M, Ws.data(), cut, P);
    for (int q = 0; q < M * M; ++q) cov[q] = P[q];
    for (int a = 0; a < M; ++a) {
        double s = 0.0;
        for (int b = 0; b < M; ++b) s += P[(size_t)a * M + b] * rhs[b];
        mean[a] = s;
    }
    double c2 = 0.0;
    for (int j = first; j < n; ++j)
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b)
                c2 += (I[(size_t)j * M + a] - mean[a]) * W[j][(size_t)a * M + b] *
                      (I[(size_t)j * M + b] - mean[b]);
    *chi2 = c2;
    return n_it;
}

// §2.5, last paragraph: with the map frozen (alpha = 0) after the first
// iterations, the unweighted mean of the I_j is unbiased, and the mean of the
// sigma_j over sqrt(N_it) estimates its error; chi^2 about that mean.
void vp::combine_unweighted(const double *I, const double *V, int n, int discard,
                            vp_result_t *r) {
    int first = discard < 0 ? 0 : discard;
    r->n_it = n > first ? n - first : 0;
    r->dof = r->n_it > 0 ? r->n_it - 1 : 0;
    r->mean = NAN;
    r->sdev = NAN;
    r->chi2 = NAN;
    if (r->n_it == 0) return;
    double si = 0.0, ss = 0.0;
    for (int j = first; j < n; ++j) {
        si += I[j];
        ss += std::sqrt(V[j] > 0.0 ? V[j] : 0.0);
    }
    r->mean = si / r->n_it;
    r->sdev = ss / r->n_it / std::sqrt((double)r->n_it);
    double c = 0.0;
    bool any_zero = false;
    for (int j = first; j < n; ++j) {
        if (V[j] > 0.0) c += (I[j] - r->mean) * (I[j] - r->mean) / V[j];
        else any_zero = true;
    }
    r->chi2 = any_zero ? 0.0 : c;
}

static vp_status member_result(Set &s, int i, int discard, vp_result_t *out,
                               bool unweighted = false) {
    CU(cudaStreamSynchronize(s.last));
    const Desc &d = s.h_desc[i];
    State st;
    CU(cudaMemcpy(&st, d.st, sizeof st, cudaMemcpyDeviceToHost));
    const int n = (int)std::min<uint32_t>(st.t, (uint32_t)d.hist_cap);
    std::vector<double> I(n), V(n);
    if (n) {
        CU(cudaMemcpy(I.data(), d.hist_i, n * 8, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(V.data(), d.hist_var, n * 8, cudaMemcpyDeviceToHost));
    }
    memset(out, 0, sizeof *out);
    if (unweighted) combine_unweighted(I.data(), V.data(), n, discard, out);
    else combine(I.data(), V.data(), n, discard, out);
    out->n_eval = (int64_t)st.n_eval_total;
    out->last_i = st.last_i;
    out->last_sdev = std::sqrt(st.last_var);
    if (st.status & kStatusNonFinite) return fail(VP_ENONFINITE, "integrand produced a non-finite value");
    return VP_OK;
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
#define CHECK_CTX(c) \
    if (!(c)) return fail(VP_EINVAL, "NULL context")

extern "C" vp_status vp_map_create(const vp_params *params, const vp_integrand *f, void *stream,
                                   vp_ctx **out) {
    if (!out) return fail(VP_EINVAL, "NULL out");
    *out = nullptr;
    vp_ctx *c = new (std::nothrow) vp_ctx();
    if (!c) return fail(VP_ENOMEM, "host allocation failed");
    vp_status st = set_create(c->set, 1, params, f, (cudaStream_t)stream);
    if (st != VP_OK) {
        std::string keep = g_err;
        set_destroy(c->set);
        delete c;
        g_err = keep;
        return st;
    }
    *out = c;
    return VP_OK;
}

extern "C" vp_status vp_iterate(vp_ctx *c, void *stream) {
    CHECK_CTX(c);
    return set_iterate(c->set, (cudaStream_t)stream);
}

extern "C" vp_status vp_adapt(vp_ctx *c, void *stream) {
    CHECK_CTX(c);
    return set_adapt(c->set, (cudaStream_t)stream);
}

extern "C" vp_status vp_step(vp_ctx *c, void *stream) {
    CHECK_CTX(c);
    return set_step(c->set, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// One integral over several devices (ranks): each samples a part of the
// iteration's samples, the parts' partial sums are added across ranks, and
// every rank then runs the same estimate and adaptation on the same sums.
// ---------------------------------------------------------------------------
static vp_status shard_check(vp_ctx *c) {
    CHECK_CTX(c);
    const Set &s = c->set;
    if (s.groups.size() != 1 || s.groups[0].blocks_plan == 0)
        return fail(VP_EINVAL, "sampling in parts needs the one-integral kernel (FP32 peak "
                               "families: at most %d peaks)", kParamPeaks);
    if (s.m[0].n_out > 1) return fail(VP_EINVAL, "sampling in parts: one output only");
    return VP_OK;
}

extern "C" vp_status vp_iterate_part(vp_ctx *c, int part, int n_parts, void *stream) {
    vp_status st = shard_check(c);
    if (st != VP_OK) return st;
    if (n_parts < 1 || n_parts > 65536 || part < 0 || part >= n_parts)
        return fail(VP_EINVAL, "part must be in 0..n_parts-1, n_parts in 1..65536");
    NvtxRange nv("vp.iterate_part");
    Set &s = c->set;
    cudaStream_t strm = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(strm, &cap));
    if (cap != cudaStreamCaptureStatusActive) {
        st = tune(s, strm);
        if (st != VP_OK) return st;
    }
    // the one-integral kernel in its tuned shape, or its planned one if the
    // tuner chose the task kernel (which has no sample ranges)
    Group g = s.groups[0];
    if (!g.one) {
        g.one = true;
        g.blocks = g.blocks_plan;
        g.cs = g.cs_plan;
        g.threads_one = g.threads_plan;
    }
    g.args1.part = part;
    g.args1.n_parts = n_parts;
    st = launch_group(s.d_desc, g, strm);
    if (st != VP_OK) return st;
    s.last = strm;
    return VP_OK;
}

extern "C" vp_status vp_partials_size(vp_ctx *c, int64_t *n) {
    CHECK_CTX(c);
    if (!n) return fail(VP_EINVAL, "NULL out");
    const Desc &d = c->set.h_desc[0];
    *n = (int64_t)(2 * d.n_hc + 2 * (uint64_t)d.dim * (uint64_t)d.n_g);
    return VP_OK;
}

static vp_status partials_move(vp_ctx *c, double *buf, int dir, cudaStream_t stream) {
    vp_status st = shard_check(c);
    if (st != VP_OK) return st;
    if (!buf) return fail(VP_EINVAL, "NULL buffer");
    cudaPointerAttributes pa;
    CU(cudaPointerGetAttributes(&pa, buf));
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
        return fail(VP_EINVAL, "the partial sums buffer must be device memory");
    int64_t n = 0;
    vp_partials_size(c, &n);
    CU(launch_partials(c->set.d_desc, buf, (uint64_t)n, dir, stream));
    c->set.last = stream;
    return VP_OK;
}

extern "C" vp_status vp_partials_export(vp_ctx *c, double *buf, void *stream) {
    return partials_move(c, buf, 0, (cudaStream_t)stream);
}

extern "C" vp_status vp_partials_import(vp_ctx *c, const double *buf, void *stream) {
    return partials_move(c, (double *)buf, 1, (cudaStream_t)stream);
}

extern "C" vp_status vp_estimate(vp_ctx *c, void *stream) {
    vp_status st = shard_check(c);
    if (st != VP_OK) return st;
    Set &s = c->set;
    CU(launch_estimate(s.d_desc, s.d_tree_base, 1, s.n_tree_total, 0, (cudaStream_t)stream,
                       set_prec(s)));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
    if (cap != cudaStreamCaptureStatusActive) ++s.iters;
    s.last = (cudaStream_t)stream;
    return VP_OK;
}

extern "C" vp_status vp_step_read(vp_ctx *c, void *stream, int *have, double *i_j,
                                  double *var_j) {
    CHECK_CTX(c);
    if (!have || !i_j || !var_j) return fail(VP_EINVAL, "NULL out");
    *have = 0;
    if (!c->pin) {
        CU(cudaHostAlloc((void **)&c->pin, 4 * sizeof(double), cudaHostAllocDefault));
        CU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (cudaEvent_t &e : c->step_ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const Desc &d = c->set.h_desc[0];
    const int64_t t = (int64_t)c->set.iters + c->t_off;  // the index of this step's iteration
    vp_status st = set_step(c->set, (cudaStream_t)stream);
    if (st != VP_OK) return st;
    const int k = c->slot;
    if (t >= 0 && t < d.hist_cap) {  // from the history, beside the next step
        CU(cudaEventRecord(c->step_ev[k], (cudaStream_t)stream));
        CU(cudaStreamWaitEvent(c->side, c->step_ev[k], 0));
        CU(cudaMemcpyAsync(c->pin + 2 * k, d.hist_i + t, sizeof(double), cudaMemcpyDeviceToHost,
                           c->side));
        CU(cudaMemcpyAsync(c->pin + 2 * k + 1, d.hist_var + t, sizeof(double),
                           cudaMemcpyDeviceToHost, c->side));
        CU(cudaEventRecord(c->ev[k], c->side));
    } else {  // the history is full: the state's copy, before the next step may change it
        const State *dst = d.st;  // last_i, last_var: adjacent doubles
        CU(cudaMemcpyAsync(c->pin + 2 * k, &dst->last_i, 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, (cudaStream_t)stream));
        CU(cudaEventRecord(c->ev[k], (cudaStream_t)stream));
    }
    if (c->pending) {  // the previous call's step, finished while this one was enqueued
        CU(cudaEventSynchronize(c->ev[k ^ 1]));
        *i_j = c->pin[2 * (k ^ 1)];
        *var_j = c->pin[2 * (k ^ 1) + 1];
        *have = 1;
    }
    c->pending = true;
    c->slot = k ^ 1;
    return VP_OK;
}

extern "C" vp_status vp_step_read_flush(vp_ctx *c, int *have, double *i_j, double *var_j) {
    CHECK_CTX(c);
    if (!have || !i_j || !var_j) return fail(VP_EINVAL, "NULL out");
    *have = 0;
    if (!c->pending) return VP_OK;
    const int k = c->slot ^ 1;
    CU(cudaEventSynchronize(c->ev[k]));
    *i_j = c->pin[2 * k];
    *var_j = c->pin[2 * k + 1];
    *have = 1;
    c->pending = false;
    return VP_OK;
}

extern "C" vp_status vp_result(vp_ctx *c, int discard, vp_result_t *out) {
    CHECK_CTX(c);
    if (!out) return fail(VP_EINVAL, "NULL out");
    return member_result(c->set, 0, discard, out);
}

extern "C" vp_status vp_result_unweighted(vp_ctx *c, int discard, vp_result_t *out) {
    CHECK_CTX(c);
    if (!out) return fail(VP_EINVAL, "NULL out");
    return member_result(c->set, 0, discard, out, true);
}

// New damping exponents for member i of a set, host and device descriptors.
static vp_status set_damping(Set &s, int i, double alpha, double beta) {
    if (!(alpha >= 0.0 && std::isfinite(alpha))) return fail(VP_EINVAL, "alpha must be finite and >= 0");
    if (!(beta >= 0.0 && std::isfinite(beta))) return fail(VP_EINVAL, "beta must be finite and >= 0");
    CU(cudaStreamSynchronize(s.last));
    Member &mb = s.m[i];
    mb.p.alpha = alpha;
    mb.p.beta = beta;
    Desc &d = s.h_desc[i];
    d.alpha = alpha;
    d.beta = beta;
    damp_consts(d, beta);
    CU(cudaMemcpy(s.d_desc + i, &d, sizeof d, cudaMemcpyHostToDevice));
    bool any = false;
    for (const Member &m : s.m) any |= m.p.alpha > 0.0 && m.p.n_g > 1;
    if (any != s.any_refine && s.gexec) {  // the step graph's shape changes: capture again
        cudaGraphExecDestroy(s.gexec);
        cudaGraphDestroy(s.graph);
        s.gexec = nullptr;
        s.graph = nullptr;
    }
    s.any_refine = any;
    return VP_OK;
}

extern "C" vp_status vp_set_damping(vp_ctx *c, double alpha, double beta) {
    CHECK_CTX(c);
    return set_damping(c->set, 0, alpha, beta);
}

extern "C" vp_status vp_map_destroy(vp_ctx *c) {
    if (!c) return VP_OK;
    if (c->pin) {
        cudaStreamSynchronize(c->set.last);
        cudaStreamSynchronize(c->side);
        cudaFreeHost(c->pin);
        cudaStreamDestroy(c->side);
    }
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->step_ev)
        if (e) cudaEventDestroy(e);
    set_destroy(c->set);
    delete c;
    return VP_OK;
}

extern "C" vp_status vp_get_info(vp_ctx *c, int64_t *n_st, int64_t *n_hc, int *n_it) {
    CHECK_CTX(c);
    CU(cudaStreamSynchronize(c->set.last));
    State st;
    CU(cudaMemcpy(&st, c->set.h_desc[0].st, sizeof st, cudaMemcpyDeviceToHost));
    if (n_st) *n_st = c->set.m[0].n_st;
    if (n_hc) *n_hc = (int64_t)c->set.m[0].n_hc;
    if (n_it) *n_it = (int)st.t;
    return VP_OK;
}

extern "C" vp_status vp_get_strata(vp_ctx *c, int32_t *strata) {
    CHECK_CTX(c);
    if (!strata) return fail(VP_EINVAL, "NULL out");
    const Member &mb = c->set.m[0];
    for (int mu = 0; mu < mb.p.dim; ++mu) strata[mu] = (int32_t)mb.nst_ax[mu];
    return VP_OK;
}

static vp_status latest_parity(Set &s, size_t *par);

// The several-outputs history of a set's member 0 (App. B): i_j[n][M], cov_j[n][M][M].
static vp_status multi_history(Set &s, int i, int n, std::vector<double> &I,
                               std::vector<double> &C) {
    const Desc &d = s.h_desc[i];
    const int M = d.n_out, T = M * (M + 1) / 2;
    std::vector<double> tri((size_t)n * T);
    I.assign((size_t)n * M, 0.0);
    C.assign((size_t)n * M * M, 0.0);
    if (n) {
        CU(cudaMemcpy(I.data(), d.hist_im, (size_t)n * M * 8, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(tri.data(), d.hist_cm, (size_t)n * T * 8, cudaMemcpyDeviceToHost));
    }
    for (int j = 0; j < n; ++j) {
        int q = 0;
        for (int k = 0; k < M; ++k)
            for (int l = k; l < M; ++l, ++q)
                C[((size_t)j * M + k) * M + l] = C[((size_t)j * M + l) * M + k] =
                    tri[(size_t)j * T + q];
    }
    return VP_OK;
}

extern "C" vp_status vp_get_history_multi(vp_ctx *c, int n, double *i_j, double *cov_j) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    if (d.n_out < 2) return fail(VP_EINVAL, "the context has no extra outputs");
    if (n < 0 || n > d.hist_cap) return fail(VP_EINVAL, "n outside the history capacity");
    CU(cudaStreamSynchronize(c->set.last));
    std::vector<double> I, C;
    vp_status st = multi_history(c->set, 0, n, I, C);
    if (st != VP_OK) return st;
    if (i_j) std::copy(I.begin(), I.end(), i_j);
    if (cov_j) std::copy(C.begin(), C.end(), cov_j);
    return VP_OK;
}

static vp_status member_result_multi(Set &s, int i, int discard, double *mean, double *cov,
                                     double *chi2, int *dof, int *n_it) {
    if (!mean || !cov || !chi2 || !dof) return fail(VP_EINVAL, "NULL out");
    const Desc &d = s.h_desc[i];
    if (d.n_out < 2) return fail(VP_EINVAL, "the integral has no extra outputs");
    CU(cudaStreamSynchronize(s.last));
    State st;
    CU(cudaMemcpy(&st, d.st, sizeof st, cudaMemcpyDeviceToHost));
    const int n = (int)std::min<uint32_t>(st.t, (uint32_t)d.hist_cap);
    std::vector<double> I, C;
    vp_status rs = multi_history(s, i, n, I, C);
    if (rs != VP_OK) return rs;
    const int used = combine_multi(I.data(), C.data(), n, d.n_out, discard, mean, cov, chi2);
    *dof = used > 0 ? d.n_out * (used - 1) : 0;
    if (n_it) *n_it = used;
    if (st.status & kStatusNonFinite) return fail(VP_ENONFINITE, "integrand produced a non-finite value");
    return VP_OK;
}

extern "C" vp_status vp_result_multi(vp_ctx *c, int discard, double *mean, double *cov,
                                     double *chi2, int *dof, int *n_it) {
    CHECK_CTX(c);
    return member_result_multi(c->set, 0, discard, mean, cov, chi2, dof, n_it);
}

extern "C" vp_status vp_get_moments_multi(vp_ctx *c, double *x1, double *x2) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    if (d.n_out < 2) return fail(VP_EINVAL, "the context has no extra outputs");
    size_t par = 0;
    vp_status st = latest_parity(c->set, &par);
    if (st != VP_OK) return st;
    const size_t M = (size_t)d.n_out, T = M * (M + 1) / 2;
    if (x1) CU(cudaMemcpy(x1, d.x1 + par * d.n_hc * M, d.n_hc * M * 8, cudaMemcpyDeviceToHost));
    if (x2) CU(cudaMemcpy(x2, d.x2 + par * d.n_hc * T, d.n_hc * T * 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}

extern "C" vp_status vp_get_edges(vp_ctx *c, double *edges) {
    CHECK_CTX(c);
    if (!edges) return fail(VP_EINVAL, "NULL edges");
    const Desc &d = c->set.h_desc[0];
    CU(cudaStreamSynchronize(c->set.last));
    CU(cudaMemcpy(edges, d.edges, (size_t)d.dim * (d.n_g + 1) * 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}

extern "C" vp_status vp_set_edges(vp_ctx *c, const double *edges) {
    CHECK_CTX(c);
    if (!edges) return fail(VP_EINVAL, "NULL edges");
    const Desc &d = c->set.h_desc[0];
    const Member &mb = c->set.m[0];
    const int D = d.dim, G = d.n_g;
    for (int mu = 0; mu < D; ++mu) {
        const double *e = edges + (size_t)mu * (G + 1);
        if (e[0] != mb.lo[mu] || e[G] != mb.hi[mu]) return fail(VP_EINVAL, "grid ends must equal the box");
        for (int k = 0; k < G; ++k)
            if (!(e[k + 1] > e[k])) return fail(VP_EINVAL, "grid must be strictly increasing");
    }
    std::vector<float2> tab((size_t)D * G);
    for (int mu = 0; mu < D; ++mu) make_tab(edges + (size_t)mu * (G + 1), G, &tab[(size_t)mu * G]);
    CU(cudaStreamSynchronize(c->set.last));
    CU(cudaMemcpy(d.edges, edges, (size_t)D * (G + 1) * 8, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(d.tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));
    return VP_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: a context's state between iterations as a byte blob.
// Layout: CkptHeader, State, edges [D][N_g + 1] f64, n_h [N_h] u32, offsets
// [N_h + 1] u64, I_j and sigma_j^2 [hist_cap] f64 each, and with extra outputs
// their history [hist_cap][M] and [hist_cap][M(M+1)/2] f64.
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];          // "vpstate1"
    uint32_t state_bytes;   // sizeof(State) of the build that wrote it
    int32_t dim, n_g, kind, prec, n_out, hist_cap, pad;
    int64_t n_ev;
    uint64_t n_hc, seed;
    uint32_t integral_id;
    int32_t strata[kMaxDim];
};

size_t ckpt_bytes(const Desc &d) {
    const size_t M = d.n_out > 1 ? (size_t)d.n_out : 0, T = M * (M + 1) / 2;
    return sizeof(CkptHeader) + sizeof(State) + (size_t)d.dim * (d.n_g + 1) * 8 + d.n_hc * 4 +
           (d.n_hc + 1) * 8 + (size_t)d.hist_cap * 16 + (size_t)d.hist_cap * (M + T) * 8;
}

CkptHeader ckpt_header(const Member &mb, const Desc &d) {
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "vpstate1", 8);
    h.state_bytes = (uint32_t)sizeof(State);
    h.dim = d.dim;
    h.n_g = d.n_g;
    h.kind = d.kind;
    h.prec = d.prec;
    h.n_out = d.n_out;
    h.hist_cap = d.hist_cap;
    h.n_ev = d.n_ev;
    h.n_hc = d.n_hc;
    h.seed = mb.p.seed;
    h.integral_id = d.integral_id;
    for (int mu = 0; mu < d.dim; ++mu) h.strata[mu] = (int32_t)mb.nst_ax[mu];
    return h;
}
}  // namespace

extern "C" vp_status vp_export_state(vp_ctx *c, void *buf, size_t cap, size_t *size) {
    CHECK_CTX(c);
    if (!size) return fail(VP_EINVAL, "NULL size");
    Set &s = c->set;
    const Desc &d = s.h_desc[0];
    const size_t need = ckpt_bytes(d);
    *size = need;
    if (!buf) return VP_OK;
    if (cap < need) return fail(VP_EINVAL, "buffer of %zu bytes, the state needs %zu", cap, need);
    CU(cudaStreamSynchronize(s.last));
    char *p = (char *)buf;
    const CkptHeader h = ckpt_header(s.m[0], d);
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    CU(cudaMemcpy(p, d.st, sizeof(State), cudaMemcpyDeviceToHost));
    p += sizeof(State);
    const size_t ne = (size_t)d.dim * (d.n_g + 1) * 8;
    CU(cudaMemcpy(p, d.edges, ne, cudaMemcpyDeviceToHost));
    p += ne;
    CU(cudaMemcpy(p, d.n_h, d.n_hc * 4, cudaMemcpyDeviceToHost));
    p += d.n_hc * 4;
    CU(cudaMemcpy(p, d.off, (d.n_hc + 1) * 8, cudaMemcpyDeviceToHost));
    p += (d.n_hc + 1) * 8;
    CU(cudaMemcpy(p, d.hist_i, (size_t)d.hist_cap * 8, cudaMemcpyDeviceToHost));
    p += (size_t)d.hist_cap * 8;
    CU(cudaMemcpy(p, d.hist_var, (size_t)d.hist_cap * 8, cudaMemcpyDeviceToHost));
    p += (size_t)d.hist_cap * 8;
    if (d.n_out > 1) {
        const size_t M = (size_t)d.n_out, T = M * (M + 1) / 2;
        CU(cudaMemcpy(p, d.hist_im, (size_t)d.hist_cap * M * 8, cudaMemcpyDeviceToHost));
        p += (size_t)d.hist_cap * M * 8;
        CU(cudaMemcpy(p, d.hist_cm, (size_t)d.hist_cap * T * 8, cudaMemcpyDeviceToHost));
    }
    return VP_OK;
}

extern "C" vp_status vp_import_state(vp_ctx *c, const void *buf, size_t size) {
    CHECK_CTX(c);
    if (!buf) return fail(VP_EINVAL, "NULL buffer");
    Set &s = c->set;
    const Desc &d = s.h_desc[0];
    const Member &mb = s.m[0];
    if (size != ckpt_bytes(d)) return fail(VP_EINVAL, "state of %zu bytes, this context's is %zu", size, ckpt_bytes(d));
    const CkptHeader want = ckpt_header(mb, d);
    CkptHeader got;
    memcpy(&got, buf, sizeof got);
    if (memcmp(&want, &got, sizeof got) != 0)
        return fail(VP_EINVAL, "the state was written by a context of other parameters");
    const char *p = (const char *)buf + sizeof(CkptHeader);
    State st;
    memcpy(&st, p, sizeof st);
    p += sizeof(State);
    const size_t ne = (size_t)d.dim * (d.n_g + 1) * 8;
    const double *edges = (const double *)p;
    for (int mu = 0; mu < d.dim; ++mu) {  // the grid as vp_set_edges checks it
        const double *e = edges + (size_t)mu * (d.n_g + 1);
        if (e[0] != mb.lo[mu] || e[d.n_g] != mb.hi[mu]) return fail(VP_EINVAL, "grid ends must equal the box");
        for (int k = 0; k < d.n_g; ++k)
            if (!(e[k + 1] > e[k])) return fail(VP_EINVAL, "grid must be strictly increasing");
    }
    std::vector<float2> tab((size_t)d.dim * d.n_g);
    for (int mu = 0; mu < d.dim; ++mu)
        make_tab(edges + (size_t)mu * (d.n_g + 1), d.n_g, &tab[(size_t)mu * d.n_g]);
    CU(cudaStreamSynchronize(s.last));
    CU(cudaMemcpy(d.edges, edges, ne, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(d.tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));
    p += ne;
    CU(cudaMemcpy(d.n_h, p, d.n_hc * 4, cudaMemcpyHostToDevice));
    p += d.n_hc * 4;
    CU(cudaMemcpy(d.off, p, (d.n_hc + 1) * 8, cudaMemcpyHostToDevice));
    p += (d.n_hc + 1) * 8;
    CU(cudaMemcpy(d.hist_i, p, (size_t)d.hist_cap * 8, cudaMemcpyHostToDevice));
    p += (size_t)d.hist_cap * 8;
    CU(cudaMemcpy(d.hist_var, p, (size_t)d.hist_cap * 8, cudaMemcpyHostToDevice));
    p += (size_t)d.hist_cap * 8;
    const size_t M = d.n_out > 1 ? (size_t)d.n_out : 0, T = M * (M + 1) / 2;
    if (M) {
        CU(cudaMemcpy(d.hist_im, p, (size_t)d.hist_cap * M * 8, cudaMemcpyHostToDevice));
        p += (size_t)d.hist_cap * M * 8;
        CU(cudaMemcpy(d.hist_cm, p, (size_t)d.hist_cap * T * 8, cudaMemcpyHostToDevice));
    }
    // both buffers of the per-iteration sums clear (either parity may come next)
    const size_t bins = (size_t)d.dim * d.n_g;
    CU(cudaMemset(d.s1, 0, 2 * d.n_hc * 8));
    CU(cudaMemset(d.s2, 0, 2 * d.n_hc * 8));
    CU(cudaMemset(d.hsum, 0, 2 * bins * 8));
    CU(cudaMemset(d.hcnt, 0, 2 * bins * 4));
    if (M) {
        CU(cudaMemset(d.x1, 0, 2 * d.n_hc * M * 8));
        CU(cudaMemset(d.x2, 0, 2 * d.n_hc * T * 8));
    }
    st.done_est = st.done_alloc = st.done_multi = 0u;
    CU(cudaMemcpy(d.st, &st, sizeof st, cudaMemcpyHostToDevice));
    c->t_off = (int64_t)st.t - (int64_t)s.iters;
    return VP_OK;
}

extern "C" vp_status vp_get_alloc(vp_ctx *c, uint32_t *n_h, uint64_t *offsets) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    CU(cudaStreamSynchronize(c->set.last));
    if (n_h) CU(cudaMemcpy(n_h, d.n_h, d.n_hc * 4, cudaMemcpyDeviceToHost));
    if (offsets) CU(cudaMemcpy(offsets, d.off, (d.n_hc + 1) * 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}

// Buffer parity of the latest iteration ((t - 1) & 1); synchronises.
static vp_status latest_parity(Set &s, size_t *par) {
    CU(cudaStreamSynchronize(s.last));
    State st;
    CU(cudaMemcpy(&st, s.h_desc[0].st, sizeof st, cudaMemcpyDeviceToHost));
    *par = (size_t)((st.t - 1u) & 1u);
    return VP_OK;
}

extern "C" vp_status vp_get_moments(vp_ctx *c, double *s1, double *s2) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    size_t par = 0;
    vp_status st = latest_parity(c->set, &par);
    if (st != VP_OK) return st;
    if (s1) CU(cudaMemcpy(s1, d.s1 + par * d.n_hc, d.n_hc * 8, cudaMemcpyDeviceToHost));
    if (s2) CU(cudaMemcpy(s2, d.s2 + par * d.n_hc, d.n_hc * 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}

extern "C" vp_status vp_get_hist(vp_ctx *c, double *hsum, double *hcnt) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    const size_t bins = (size_t)d.dim * d.n_g;
    size_t par = 0;
    vp_status st = latest_parity(c->set, &par);
    if (st != VP_OK) return st;
    if (hsum) CU(cudaMemcpy(hsum, d.hsum + par * bins, bins * 8, cudaMemcpyDeviceToHost));
    if (hcnt) {
        std::vector<uint32_t> tmp(bins);
        CU(cudaMemcpy(tmp.data(), d.hcnt + par * bins, bins * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < bins; ++i) hcnt[i] = (double)tmp[i];
    }
    return VP_OK;
}

extern "C" vp_status vp_get_dh(vp_ctx *c, double *d_h, double *sum_d) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    CU(cudaStreamSynchronize(c->set.last));
    if (d_h) CU(cudaMemcpy(d_h, d.dh, d.n_hc * 8, cudaMemcpyDeviceToHost));
    if (sum_d) CU(cudaMemcpy(sum_d, &d.st->sum_d, 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}

extern "C" vp_status vp_get_history(vp_ctx *c, int n, double *i_j, double *var_j) {
    CHECK_CTX(c);
    const Desc &d = c->set.h_desc[0];
    if (n < 0 || n > d.hist_cap) return fail(VP_EINVAL, "n outside the history capacity");
    CU(cudaStreamSynchronize(c->set.last));
    if (n && i_j) CU(cudaMemcpy(i_j, d.hist_i, n * 8, cudaMemcpyDeviceToHost));
    if (n && var_j) CU(cudaMemcpy(var_j, d.hist_var, n * 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}

static vp_status alloc_from(vp_ctx *c, const double *v, int mode, cudaStream_t stream) {
    CHECK_CTX(c);
    if (!v) return fail(VP_EINVAL, "NULL input");
    Set &s = c->set;
    const Desc &d = s.h_desc[0];
    for (uint64_t h = 0; h < d.n_hc; ++h)
        if (!(v[h] >= 0.0) || !std::isfinite(v[h])) return fail(VP_EINVAL, "entries must be finite and >= 0");
    CU(cudaStreamSynchronize(s.last));
    CU(cudaMemcpyAsync(d.dh, v, d.n_hc * 8, cudaMemcpyHostToDevice, stream));
    CU(launch_estimate(s.d_desc, s.d_tree_base, 1, s.n_tree_total, mode, stream, set_prec(s)));
    CU(launch_alloc(s.d_desc, s.d_tree_base, 1, s.n_tree_total, stream, 0));
    CU(cudaStreamSynchronize(stream));
    s.last = stream;
    return VP_OK;
}

extern "C" vp_status vp_alloc_from_dh(vp_ctx *c, const double *d_h, void *stream) {
    return alloc_from(c, d_h, 2, (cudaStream_t)stream);
}

extern "C" vp_status vp_alloc_from_sigma(vp_ctx *c, const double *sigma_h, void *stream) {
    return alloc_from(c, sigma_h, 1, (cudaStream_t)stream);
}

extern "C" vp_status vp_refine_from_hist(vp_ctx *c, const double *hsum, const double *hcnt,
                                         void *stream) {
    CHECK_CTX(c);
    if (!hsum || !hcnt) return fail(VP_EINVAL, "NULL histogram");
    Set &s = c->set;
    const Desc &d = s.h_desc[0];
    const size_t bins = (size_t)d.dim * d.n_g;
    std::vector<uint32_t> cnt(bins);
    for (size_t i = 0; i < bins; ++i) {
        if (!(hcnt[i] >= 0.0 && hcnt[i] < 4294967296.0) || hcnt[i] != std::floor(hcnt[i]))
            return fail(VP_EINVAL, "counts must be integers in [0, 2^32)");
        if (!std::isfinite(hsum[i]) || hsum[i] < 0.0) return fail(VP_EINVAL, "sums must be finite and >= 0");
        cnt[i] = (uint32_t)hcnt[i];
    }
    size_t par = 0;  // the refinement reads the latest iteration's buffer
    vp_status pst = latest_parity(s, &par);
    if (pst != VP_OK) return pst;
    CU(cudaMemcpyAsync(d.hsum + par * bins, hsum, bins * 8, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CU(cudaMemcpyAsync(d.hcnt + par * bins, cnt.data(), bins * 4, cudaMemcpyHostToDevice,
                       (cudaStream_t)stream));
    // (the sums are taken as the context accumulates them: weighted or plain)
    const uint32_t par32 = (uint32_t)par | (d.d_weighted ? 2u : 0u);
    CU(cudaMemcpyAsync((char *)d.st + offsetof(State, hist_par), &par32, 4, cudaMemcpyHostToDevice,
                       (cudaStream_t)stream));
    CU(launch_refine(s.d_desc, s.d_axis_base, 1, s.n_axis_total, s.max_ng, (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    s.last = (cudaStream_t)stream;
    return VP_OK;
}

extern "C" vp_status vp_precondition(vp_ctx *c, int64_t n, const double *x, const double *f,
                                     int n_iter, void *stream) {
    CHECK_CTX(c);
    NvtxRange nv("vp.precondition");
    Set &s = c->set;
    const Member &mb = s.m[0];
    const Desc &d = s.h_desc[0];
    const int D = mb.p.dim;
    if (n < 1 || !x) return fail(VP_EINVAL, "need at least one data point");
    if (n_iter < 0) return fail(VP_EINVAL, "n_iter must be >= 0");
    for (int64_t p = 0; p < n; ++p) {
        for (int mu = 0; mu < D; ++mu) {
            const double v = x[p * D + mu];
            if (!(v >= mb.lo[mu] && v <= mb.hi[mu]))
                return fail(VP_EINVAL, "data point %lld outside the box on axis %d", (long long)p, mu);
        }
        if (f && !std::isfinite(f[p])) return fail(VP_EINVAL, "non-finite f at data point %lld", (long long)p);
    }
    if (n_iter == 0) return VP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    size_t par = 0;  // the previous iteration's histogram buffer: the next estimate clears it
    vp_status pst = latest_parity(s, &par);
    if (pst != VP_OK) return pst;
    const size_t bins = (size_t)D * d.n_g;
    DevMem tmp;
    const size_t xb = align256((size_t)n * D * 8);
    vp_status ast = dev_alloc(tmp, xb + (f ? (size_t)n * 8 : 0), st);
    if (ast != VP_OK) return ast;
    double *dx = (double *)tmp.ptr;
    double *df = f ? (double *)((char *)tmp.ptr + xb) : nullptr;
    const uint32_t par32 = (uint32_t)par;
    cudaError_t e = cudaMemcpyAsync(dx, x, (size_t)n * D * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(df, f, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char *)d.st + offsetof(State, hist_par), &par32, 4,
                            cudaMemcpyHostToDevice, st);
    for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
        e = cudaMemsetAsync(d.hsum + par * bins, 0, bins * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.hcnt + par * bins, 0, bins * 4, st);
        if (e == cudaSuccess)
            e = launch_precondition(mb.bucket, mb.kind, st, s.d_desc, 0, n, dx, df, par32);
        if (e == cudaSuccess)
            e = launch_refine(s.d_desc, s.d_axis_base, 1, s.n_axis_total, s.max_ng, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(tmp, st);
    cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(VP_ECUDA, "vp_precondition: %s", cudaGetErrorString(e));
    s.last = st;
    return VP_OK;
}

extern "C" vp_status vp_eval_samples(vp_ctx *c, int64_t n, const uint64_t *h, const uint32_t *j,
                                     uint32_t t, double *x, int32_t *idx, double *jac, double *f) {
    CHECK_CTX(c);
    if (n < 0) return fail(VP_EINVAL, "n < 0");
    if (n == 0) return VP_OK;
    if (!h || !j || !x || !idx || !jac || !f) return fail(VP_EINVAL, "NULL buffer");
    Set &s = c->set;
    const Desc &d = s.h_desc[0];
    for (int64_t k = 0; k < n; ++k)
        if (h[k] >= d.n_hc) return fail(VP_EINVAL, "hypercube index %llu out of range", (unsigned long long)h[k]);
    const size_t D = d.dim;
    const size_t bytes = n * (8 + 4 + D * 8 + D * 4 + 8 + 8) + 6 * 256;
    DevMem tmp;
    cudaStream_t stream = s.last;
    CU(cudaStreamSynchronize(stream));
    vp_status st = dev_alloc(tmp, bytes, stream);
    if (st != VP_OK) return st;
    char *p = (char *)tmp.ptr;
    uint64_t *dh_ = (uint64_t *)p;
    p += align256(n * 8);
    uint32_t *dj = (uint32_t *)p;
    p += align256(n * 4);
    double *dx = (double *)p;
    p += align256(n * D * 8);
    int32_t *di = (int32_t *)p;
    p += align256(n * D * 4);
    double *djac = (double *)p;
    p += align256(n * 8);
    double *df = (double *)p;
    cudaError_t e = cudaMemcpyAsync(dh_, h, n * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dj, j, n * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = d.prec == VP_FP64
                ? launch_eval_f64(s.m[0].bucket, false, d.kind, stream, s.d_desc, 0, n, dh_, dj, t, dx, di,
                                  djac, df, 0)
                : launch_eval_f32(s.m[0].bucket, s.m[0].exact, d.kind, stream, s.d_desc, 0, n, dh_, dj, t,
                                  dx, di, djac, df, (int)((s.m[0].prm32.size() + 3) & ~(size_t)3));
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, dx, n * D * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, di, n * D * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(jac, djac, n * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, df, n * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    dev_free(tmp, stream);
    cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(VP_ECUDA, "vp_eval_samples: %s", cudaGetErrorString(e));
    return VP_OK;
}

extern "C" vp_status vp_last_sample_ms(vp_ctx *c, float *ms) {
    CHECK_CTX(c);
    if (!ms) return fail(VP_EINVAL, "NULL out");
    *ms = -1.0f;
    if (!c->set.timed) return VP_OK;
    CU(cudaEventSynchronize(c->set.ev1));
    CU(cudaEventElapsedTime(ms, c->set.ev0, c->set.ev1));
    return VP_OK;
}

extern "C" vp_status vp_get_tuning(vp_ctx *c, int *scheme, int *blocks, int *threads,
                                    int *cluster, int *run) {
    CHECK_CTX(c);
    if (c->set.groups.empty()) return fail(VP_EINVAL, "no sampling group");
    const Group &g = c->set.groups[0];
    if (scheme) *scheme = g.one ? (g.static16 >= 16 ? 0 : 2) : 1;
    if (blocks) *blocks = g.blocks;
    if (threads) *threads = g.one ? g.threads_one : g.threads;
    if (cluster) *cluster = g.cs;
    if (run) *run = g.r;
    return VP_OK;
}

extern "C" vp_status vp_set_tuning(vp_ctx *c, int scheme, int blocks, int threads, int cluster,
                                    int run) {
    CHECK_CTX(c);
    if (c->set.groups.empty()) return fail(VP_EINVAL, "no sampling group");
    Group &g = c->set.groups[0];
    if (scheme < 0 || scheme > 2) return fail(VP_EINVAL, "scheme must be 0, 1 or 2");
    const int static16 = scheme == 2 ? kTailShare : kStaticShare;
    if (scheme == 2) scheme = 0;  // the one-integral kernel with a dynamic tail
    if (scheme == 1 && threads != 256) return fail(VP_EINVAL, "the task scheme runs 256 threads");
    if (threads != 256 && threads != 512 && threads != 768 && threads != 1024)
        return fail(VP_EINVAL, "threads must be 256, 512, 768 or 1024");
    if (threads > one_max_threads(bucket_dim(g.bucket), g.prec == VP_FP64, g.p1))
        return fail(VP_EINVAL, "%d threads exceed this kernel's largest CTA", threads);
    if (scheme == 0 && g.members.size() == 1 && g.prec == VP_FP32 && g.kind != VP_POSTERIOR &&
        (int)c->set.m[g.members[0]].prm[0] > kParamPeaks)
        return fail(VP_EINVAL, "more than %d peaks: the task scheme only", kParamPeaks);
    if (blocks < 1 || blocks > 65535) return fail(VP_EINVAL, "blocks out of range");
    if (run < 1 || run > 64) return fail(VP_EINVAL, "run must be in 1..64");
    if (scheme == 1 && cluster != 1) return fail(VP_EINVAL, "the task scheme takes no clusters");
    if (scheme == 1 && !g.uniform && g.exact)
        return fail(VP_EINVAL, "strata that differ between axes at this exact dimension: the "
                               "one-integral scheme only");
    if (scheme == 1 && g.mo) return fail(VP_EINVAL, "several outputs: the one-integral scheme only");
    if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8)
        return fail(VP_EINVAL, "cluster must be 1, 2, 4 or 8");
    if (cluster > 1 && !(scheme == 0 ? g.hist_one : g.hist_shared))
        return fail(VP_EINVAL, "clusters need shared-memory histograms");
    if (blocks % cluster) return fail(VP_EINVAL, "blocks must be a multiple of the cluster");
    if (scheme == 0) {
        // the static split assumes every CTA resident at once
        const int occ = g.prec == VP_FP64
                            ? sample_occupancy_f64(g.bucket, g.exact, g.kind, true, threads, g.smem_one, g.mo)
                            : sample_occupancy_f32(g.bucket, g.exact, g.kind, true, threads, g.smem_one, false, g.p1);
        const int res = cluster > 1
                            ? (g.prec == VP_FP64
                                   ? sample_cluster_ctas_f64(g.bucket, g.exact, g.kind, cluster, blocks, threads, g.smem_one, g.mo)
                                   : sample_cluster_ctas_f32(g.bucket, g.exact, g.kind, cluster, blocks, threads, g.smem_one, g.p1))
                            : occ * c->set.n_sm;
        if (blocks > res)
            return fail(VP_EINVAL, "%d CTAs in clusters of %d exceed the %d resident ones", blocks,
                        cluster, res);
    }
    CU(cudaStreamSynchronize(c->set.last));
    if (c->set.gexec) {  // the step graph holds the old shape: capture again
        cudaGraphExecDestroy(c->set.gexec);
        cudaGraphDestroy(c->set.graph);
        c->set.gexec = nullptr;
        c->set.graph = nullptr;
    }
    g.one = scheme == 0;
    g.blocks = blocks;
    g.cs = cluster;
    g.r = run;
    g.threads_one = threads;
    g.static16 = static16;
    g.tuned_final = true;
    g.args1.r = run;
    g.args1.static16 = static16;
    double expect = 0.0;
    for (uint32_t i : g.members) expect += (double)c->set.m[i].p.n_ev + 2.0 * (double)c->set.m[i].n_hc;
    set_task(g, expect);
    g.tuned = true;
    return VP_OK;
}

// ---------------------------------------------------------------------------
// Batches: many independent integrals iterated together
// ---------------------------------------------------------------------------
#define CHECK_BATCH(b) \
    if (!(b)) return fail(VP_EINVAL, "NULL batch")

extern "C" vp_status vp_batch_create(int n, const vp_params *params, const vp_integrand *fs,
                                     void *stream, vp_batch **out) {
    if (!out) return fail(VP_EINVAL, "NULL out");
    *out = nullptr;
    if (n < 1 || n > (1 << 20)) return fail(VP_EINVAL, "batch size must be 1..1048576");
    vp_batch *b = new (std::nothrow) vp_batch();
    if (!b) return fail(VP_ENOMEM, "host allocation failed");
    b->set.merge = true;
    vp_status st = set_create(b->set, n, params, fs, (cudaStream_t)stream);
    if (st != VP_OK) {
        std::string keep = g_err;
        set_destroy(b->set);
        delete b;
        g_err = keep;
        return st;
    }
    *out = b;
    return VP_OK;
}

extern "C" vp_status vp_batch_iterate(vp_batch *b, void *stream) {
    CHECK_BATCH(b);
    return set_iterate(b->set, (cudaStream_t)stream);
}

extern "C" vp_status vp_batch_adapt(vp_batch *b, void *stream) {
    CHECK_BATCH(b);
    return set_adapt(b->set, (cudaStream_t)stream);
}

extern "C" vp_status vp_batch_step(vp_batch *b, void *stream) {
    CHECK_BATCH(b);
    return set_step(b->set, (cudaStream_t)stream);
}

extern "C" vp_status vp_batch_result(vp_batch *b, int i, int discard, vp_result_t *out) {
    CHECK_BATCH(b);
    if (!out) return fail(VP_EINVAL, "NULL out");
    if (i < 0 || i >= (int)b->set.m.size()) return fail(VP_EINVAL, "integral index out of range");
    return member_result(b->set, i, discard, out);
}

extern "C" vp_status vp_batch_results(vp_batch *b, int discard, vp_result_t *out) {
    CHECK_BATCH(b);
    if (!out) return fail(VP_EINVAL, "NULL out");
    Set &s = b->set;
    CU(cudaStreamSynchronize(s.last));
    vp_status worst = VP_OK;
    for (int i = 0; i < (int)s.m.size(); ++i) {
        vp_status st = member_result(s, i, discard, out + i);
        if (st != VP_OK && worst == VP_OK) worst = st;
    }
    return worst;
}

extern "C" vp_status vp_batch_size(vp_batch *b, int *n) {
    CHECK_BATCH(b);
    if (!n) return fail(VP_EINVAL, "NULL out");
    *n = (int)b->set.m.size();
    return VP_OK;
}

extern "C" vp_status vp_batch_destroy(vp_batch *b) {
    if (!b) return VP_OK;
    set_destroy(b->set);
    delete b;
    return VP_OK;
}

extern "C" vp_status vp_batch_result_multi(vp_batch *b, int i, int discard, double *mean,
                                           double *cov, double *chi2, int *dof, int *n_it) {
    CHECK_BATCH(b);
    if (i < 0 || i >= (int)b->set.m.size()) return fail(VP_EINVAL, "integral index out of range");
    return member_result_multi(b->set, i, discard, mean, cov, chi2, dof, n_it);
}

extern "C" vp_status vp_batch_history_multi(vp_batch *b, int i, int n, double *i_j,
                                            double *cov_j) {
    CHECK_BATCH(b);
    if (i < 0 || i >= (int)b->set.m.size()) return fail(VP_EINVAL, "integral index out of range");
    const Desc &d = b->set.h_desc[i];
    if (d.n_out < 2) return fail(VP_EINVAL, "the integral has no extra outputs");
    if (n < 0 || n > d.hist_cap) return fail(VP_EINVAL, "n outside the history capacity");
    CU(cudaStreamSynchronize(b->set.last));
    std::vector<double> I, C;
    vp_status st = multi_history(b->set, i, n, I, C);
    if (st != VP_OK) return st;
    if (i_j) std::copy(I.begin(), I.end(), i_j);
    if (cov_j) std::copy(C.begin(), C.end(), cov_j);
    return VP_OK;
}

extern "C" vp_status vp_batch_history(vp_batch *b, int i, int n, double *i_j, double *var_j) {
    CHECK_BATCH(b);
    if (i < 0 || i >= (int)b->set.m.size()) return fail(VP_EINVAL, "integral index out of range");
    const Desc &d = b->set.h_desc[i];
    if (n < 0 || n > d.hist_cap) return fail(VP_EINVAL, "n outside the history capacity");
    CU(cudaStreamSynchronize(b->set.last));
    if (n && i_j) CU(cudaMemcpy(i_j, d.hist_i, n * 8, cudaMemcpyDeviceToHost));
    if (n && var_j) CU(cudaMemcpy(var_j, d.hist_var, n * 8, cudaMemcpyDeviceToHost));
    return VP_OK;
}
