// host.h -- host-side internals shared by the translation units of libvegasp
// (the context/batch API in api.cu and the request server in server.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sample_impl.cuh"
#include "vp_internal.cuh"

#include <nvtx3/nvToolsExt.h>

namespace vp {

// A named NVTX range over a host call (shown by profilers; free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


// kernel launchers (adapt.cu)
cudaError_t launch_chunks(const Desc *, const uint32_t *, int, uint64_t *, uint32_t *, uint32_t,
                          cudaStream_t);
// (prec: VP_FP32 or VP_FP64 when every integral of the launch takes that path, else -1)
cudaError_t launch_estimate(const Desc *, const uint32_t *, int, uint32_t, int, cudaStream_t,
                            int prec = -1);
cudaError_t launch_estimate_multi(const Desc *, uint32_t, cudaStream_t);
cudaError_t launch_alloc(const Desc *, const uint32_t *, int, uint32_t, cudaStream_t, int initial);
cudaError_t launch_refine(const Desc *, const uint32_t *, int, uint32_t, int, cudaStream_t);
cudaError_t launch_partials(const Desc *, double *, uint64_t, int dir, cudaStream_t);


// the calling thread's last error message (vp_last_error)
extern thread_local std::string g_err;
vp_status fail(vp_status s, const char *fmt, ...);

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::vp::fail(VP_ECUDA, "%s failed: %s (%s:%d)", #call,                 \
                              cudaGetErrorString(e_), __FILE__, __LINE__);              \
    } while (0)

// Device memory through the allocator set by vp_set_allocator, else
// cudaMallocAsync on the given stream.
struct DevMem {
    void *ptr = nullptr;
    size_t bytes = 0;
    vp_alloc_fn alloc = nullptr;
    vp_free_fn free_fn = nullptr;
    void *user = nullptr;
};
vp_status dev_alloc(DevMem &m, size_t bytes, cudaStream_t s);
void dev_free(DevMem &m, cudaStream_t s);

// One integral: validated parameters, derived sizes and where its buffers sit.
struct Member {
    vp_params p;
    int kind;
    std::vector<double> lo, hi, prm;
    std::vector<float> prm32;
    int64_t n_st;                 // the smallest of nst_ax
    std::vector<int64_t> nst_ax;  // strata per axis (§3.2)
    bool uniform;                 // every axis has n_st strata
    int n_out = 1;                // outputs integrated on the same samples (App. B)
    std::vector<int32_t> mono;    // [2 n_out] factors (a, b) of g_k = x^a x^b; output 0 (-1, -1)
    uint64_t n_hc;
    uint32_t n_tree;
    int hist_cap;
    int bucket;
    bool exact;            // dim equals the bucket's dimension
    char *base = nullptr;  // device memory the offsets below are relative to
    size_t off_bytes[24];  // offsets of the buffers from base
};

// One sampling launch: the integrals of one kernel instantiation.
// the one-integral kernel's share of samples split statically, in 16ths: all
// of them by default; half with a dynamic tail (launch scheme 2)
constexpr int kStaticShare = 16, kTailShare = 8;

struct Group {
    int bucket, kind, prec;
    bool exact;
    std::vector<uint32_t> members;
    uint32_t *d_members = nullptr;
    uint64_t *d_chunk_base = nullptr;
    uint32_t *d_head = nullptr;      // d_head[0] queue head, d_head[1] exit counter
    int threads = 256, r = 8, blocks = 1, hist_shared = 0, hist_words = 0, prm_words = 0;
    uint32_t task = 0;
    size_t smem = 0;
    bool one = false;  // a single integral: the cluster kernel with constants in parameters
    bool uniform = true;  // every member has the same strata on every axis (else: one only)
    bool mo = false;      // several outputs (App. B): the FP64 one-integral kernel that sums them
    bool solo = false;    // a group of one member by construction (several outputs)
    bool p1 = false;      // the one-integral kernel's single-peak FP32 form
    int cs = 1;        // CTAs per cluster (one-integral kernel)
    int threads_one = 256;  // CTA size of the one-integral kernel
    // the one-integral kernel's static share of the samples in 16ths (16: all;
    // the rest pulled by warps in chunks of 32 r samples)
    int static16 = kStaticShare;
    // the one-integral kernel's shape as planned (before the autotuner), for
    // launches that need that kernel whatever the tuner chose (sharded sampling)
    int blocks_plan = 0, cs_plan = 1, threads_plan = 256;
    // histograms of the one-integral kernel (one CTA per SM fits more shared
    // memory than the task kernel's two): kHist* mode and dynamic shared bytes
    int hist_one = 0;
    size_t smem_one = 0;
    SampleOne args1;
    int occ_one = 0, occ_many = 0;  // resident CTAs per SM of each kernel
    bool tuned = false;
    // tuned on an adapted state (or fixed by the caller): the first tuning runs
    // on the uniform grid of iteration 0, whose costs differ from later ones,
    // so the shape is measured once more after kRetuneIt iterations
    bool tuned_final = false;
};
constexpr int kRetuneIt = 4;

enum {
    B_EDGES, B_TAB, B_PRM, B_PRM32, B_NH, B_OFF, B_S1, B_S2, B_DH, B_HSUM, B_HCNT, B_PART,
    B_BSUM, B_HI, B_HV, B_ST, B_X1, B_X2, B_MPART, B_HIM, B_HCM, B_COUNT
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
T *mbuf(const Member &mb, int which) {
    return (T *)(mb.base + mb.off_bytes[which]);
}

int bucket_of(int dim);
// Checks one integral's parameters and fills the host side of a Member.
vp_status validate(const vp_params *p, const vp_integrand *f, Member &mb);
// Lays out the member's buffers from byte offset `base`; returns the end.
size_t member_layout(Member &mb, size_t base);
// The member's descriptor (mb.base must be set).
void fill_desc(const Member &mb, const double *d_inv, Desc &d);
// Uniform grid, its FP32 mirror, the integrand blobs, d_h = 1 and the initial
// state, copied to the member's (zeroed) buffers on `stream`.
vp_status upload_member_init(const Member &mb, const Desc &d, cudaStream_t stream);
// Table for n < kInvTab (host arithmetic), for the descriptors, 32 bytes per
// n: 1/n and 1/(n (n-1)) (IEEE divisions), log2 n as a float pair hi + lo.
void inv_table(std::vector<double> &inv);
// The FP32 path's constants of the damping power beta in a descriptor (n_hc set).
void damp_consts(Desc &d, double beta);
// Shared memory and residency of a task-kernel group from its members.
// (g.members index m)
vp_status group_config_many(const std::vector<const Member *> &m, Group &g, int n_sm);
// Size of the tasks for `expect` samples over the group's blocks.
void set_task(Group &g, double expect);
// One sampling launch of a group.
vp_status launch_group(const Desc *d_desc, Group &g, cudaStream_t stream);
// §2.5 combination of iterations j >= discard.
void combine(const double *I, const double *V, int n, int discard, vp_result_t *r);
// §2.5 unweighted combination (frozen map) of iterations j >= discard.
void combine_unweighted(const double *I, const double *V, int n, int discard, vp_result_t *r);
// Several integrals (App. B) over iterations j >= discard: I[n][M], C[n][M][M];
// mean[M], cov[M][M], chi2, dof = M (n_it - 1).  Returns the iterations used.
int combine_multi(const double *I, const double *C, int n, int M, int discard, double *mean,
                  double *cov, double *chi2);

}  // namespace vp
