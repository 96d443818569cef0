// exa_api.cu -- the C ABI of include/exa.h: model creation (validation, NVRTC compilation of the
// generated kernels, upload, device structure pass and sorts) and the evaluation callbacks.
//
// Evaluation data flow (Sec. 5.3, 7.2.3):
//   eval kernel (generated; one thread per pattern instance, one CTA per tile of BLOCK instances of
//   one (member, pattern) pair) writes every COO slot exactly once, constraint base values
//   c[row], augmentation terms, objective gradient slots and one objective partial per CTA;
//   then atomic-free gather kernels sum duplicates: dense gradient per variable, augmentation terms
//   per row, CSC values per (row, col), the objective partials, and the products.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "exa_internal.h"

cudaError_t exa_sort_pairs_u64(const unsigned long long *kin, unsigned long long *kout, const int *vin,
                               int *vout, int n, int end_bit, cudaStream_t s);
cudaError_t exa_inclusive_sum_i32(const int *in, int *out, int n, cudaStream_t s);

using exa::Mode;
typedef long long i64;

// ------------------------------------------------------------------ static kernels
namespace {

// f[0] = sum of the per-CTA objective partials in a fixed order (deterministic for a given n and
// block size; launched with one CTA of 1024 threads, so 32 warp sums are added by thread 0).
__global__ void __launch_bounds__(1024) k_obj_final(const double *__restrict__ part, int n, double *__restrict__ f) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        f[0] = t;
    }
}

// The gathers below are latency-bound unless each thread keeps several independent loads in
// flight: a gather is an index load followed by a dependent value load, so EXA_ILP of them are
// issued back to back (indices first, then values) before any result is used.
#define EXA_ILP 8

// Segmented gather-sums, no atomics: for segment s < n, the values src[perm[q]] for q in
// [ptr[s], ptr[s+1]) are added in ascending q starting from 0.0 (ROWS: from dst[rows[s]]), and the
// result is stored to dst[s] (ROWS: dst[rows[s]]).  One warp takes 32 x EXA_SEG_G consecutive
// segments, whose entries are one contiguous range of sorted positions: all lanes gather that range
// in chunks of EXA_SEG_CHUNK into shared memory (EXA_ILP independent index-then-value loads per
// lane), then every lane adds up its own EXA_SEG_G segments from shared memory.
#define EXA_SEG_CHUNK 256
#define EXA_SEG_G 2
template <bool ROWS>
__global__ void __launch_bounds__(256) k_seg_sum_warp(const int *__restrict__ ptr, const int *__restrict__ perm,
                                                      const double *__restrict__ src, double *__restrict__ dst,
                                                      const int *__restrict__ rows, int n) {
    __shared__ double buf[8][EXA_SEG_CHUNK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long s0 = ((long long)blockIdx.x * 8 + w) * (32 * EXA_SEG_G);
    if (s0 >= n) return;
    const int beg = ptr[s0], end = ptr[min((long long)n, s0 + 32 * EXA_SEG_G)];
    int myb[EXA_SEG_G], mye[EXA_SEG_G], row[EXA_SEG_G];
    double acc[EXA_SEG_G];
#pragma unroll
    for (int g = 0; g < EXA_SEG_G; g++) {
        const long long s = s0 + 32 * g + lane;
        myb[g] = s < n ? ptr[s] : end;
        mye[g] = s < n ? ptr[s + 1] : end;
        row[g] = ROWS && s < n ? rows[s] : 0;
        acc[g] = ROWS && s < n ? dst[row[g]] : 0.0;
    }
    for (int c0 = beg; c0 < end; c0 += EXA_SEG_CHUNK) {
        const int c1 = min(c0 + EXA_SEG_CHUNK, end);
        int p[EXA_ILP];
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++) {
            const int e = c0 + lane + 32 * u;
            p[u] = e < c1 ? __ldg(perm + e) : -1;
        }
        double v[EXA_ILP];
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++) v[u] = p[u] >= 0 ? __ldg(src + p[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++)
            if (p[u] >= 0) buf[w][lane + 32 * u] = v[u];
        __syncwarp();
#pragma unroll
        for (int g = 0; g < EXA_SEG_G; g++) {
            const int qb = max(myb[g], c0), qe = min(mye[g], c1);
            for (int q = qb; q < qe; q++) acc[g] += buf[w][q - c0];
        }
        __syncwarp();
    }
#pragma unroll
    for (int g = 0; g < EXA_SEG_G; g++) {
        const long long s = s0 + 32 * g + lane;
        if (s < n) dst[ROWS ? (long long)row[g] : s] = acc[g];
    }
}

// out[i] = sum_{q in [ptr[i], ptr[i+1])} val[perm[q]] * v[other[perm[q]]], q ascending; one warp per
// 32 consecutive segments with the products of the warp's range gathered into shared memory by all
// lanes first (the k_seg_sum_warp scheme).
__global__ void __launch_bounds__(256) k_spmv_warp(const int *__restrict__ ptr, const int *__restrict__ perm,
                                                   const double *__restrict__ val, const int *__restrict__ other,
                                                   const double *__restrict__ v, double *__restrict__ out, int n) {
    __shared__ double buf[8][EXA_SEG_CHUNK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long s0 = ((long long)blockIdx.x * 8 + w) * 32;
    if (s0 >= n) return;
    const int s = (int)s0 + lane;
    const bool valid = s < n;
    const int beg = ptr[s0], end = ptr[min((long long)n, s0 + 32)];
    const int myb = valid ? ptr[s] : end, mye = valid ? ptr[s + 1] : end;
    double acc = 0.0;
    for (int c0 = beg; c0 < end; c0 += EXA_SEG_CHUNK) {
        const int c1 = min(c0 + EXA_SEG_CHUNK, end);
        int p[EXA_ILP], o[EXA_ILP];
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++) {
            const int e = c0 + lane + 32 * u;
            p[u] = e < c1 ? __ldg(perm + e) : -1;
        }
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++) o[u] = p[u] >= 0 ? __ldg(other + p[u]) : 0;
        double a[EXA_ILP], b[EXA_ILP];
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++) {
            a[u] = p[u] >= 0 ? __ldg(val + p[u]) : 0.0;
            b[u] = p[u] >= 0 ? __ldg(v + o[u]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < EXA_ILP; u++)
            if (p[u] >= 0) buf[w][lane + 32 * u] = a[u] * b[u];
        __syncwarp();
        const int qb = max(myb, c0), qe = min(mye, c1);
        for (int q = qb; q < qe; q++) acc += buf[w][q - c0];
        __syncwarp();
    }
    if (valid) out[s] = acc;
}

// dst[i] = src[perm[i]]  (CSC of a COO pattern without duplicate entries: a pure permutation).
// A block covers EXA_ILP x 256 consecutive positions; thread t takes positions t, t + 256, ... so
// that the index loads and the stores stay coalesced.
__global__ void __launch_bounds__(256) k_permute(const int *__restrict__ perm, const double *__restrict__ src,
                                                 double *__restrict__ dst, long long n) {
    const long long i0 = (long long)blockIdx.x * (256 * EXA_ILP) + threadIdx.x;
    int p[EXA_ILP];
#pragma unroll
    for (int u = 0; u < EXA_ILP; u++) p[u] = i0 + 256 * u < n ? __ldg(perm + i0 + 256 * u) : -1;
    double v[EXA_ILP];
#pragma unroll
    for (int u = 0; u < EXA_ILP; u++) v[u] = p[u] >= 0 ? __ldg(src + p[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < EXA_ILP; u++)
        if (p[u] >= 0) dst[i0 + 256 * u] = v[u];
}

// Hv[i] from the lower-triangle CSC values: column i holds (r, i), r >= i, giving H_ir v_r; the
// row-sorted permutation lists the entries (i, c), c < i, giving H_ic v_c.
__global__ void k_hprod_csc(const int *__restrict__ colptr, const int *__restrict__ rowval,
                            const double *__restrict__ val, const int *__restrict__ rptr,
                            const int *__restrict__ rperm, const int *__restrict__ colof,
                            const double *__restrict__ v, double *__restrict__ out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int p = colptr[i], e = colptr[i + 1]; p < e; p++) s += val[p] * v[rowval[p]];
    for (int q = rptr[i], e = rptr[i + 1]; q < e; q++) {
        const int p = rperm[q], c = colof[p];
        if (c != i) s += val[p] * v[c];
    }
    out[i] = s;
}

// colof[p] = column of CSC position p
__global__ void k_col_of(const int *__restrict__ colptr, int *colof, int ncol) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    for (int p = colptr[c], e = colptr[c + 1]; p < e; p++) colof[p] = c;
}

// ---- setup kernels
__global__ void k_iota(int *a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}
__global__ void k_keys2(const int *__restrict__ hi, const int *__restrict__ lo, unsigned long long *k, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = ((unsigned long long)(unsigned)hi[i] << 32) | (unsigned)(lo ? lo[i] : 0);
}
__global__ void k_keys1(const int *__restrict__ a, unsigned long long *k, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = (unsigned long long)(unsigned)a[i];
}
__global__ void k_new_segment(const unsigned long long *__restrict__ k, int *flag, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}
// segment s starts at sorted position segptr[s]; its key is segkey[s]; every sorted position's
// original index perm[i] maps to its segment in coo2seg (optional)
__global__ void k_segments(const unsigned long long *__restrict__ k, const int *__restrict__ flag,
                           const int *__restrict__ segid, const int *__restrict__ perm, int *segptr,
                           unsigned long long *segkey, int *coo2seg, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = segid[i] - 1;
    if (coo2seg) coo2seg[perm[i]] = s;
    if (flag[i]) {
        segptr[s] = i;
        segkey[s] = k[i];
    }
    if (i == n - 1) segptr[s + 1] = n;
}
// ptr[c] = first position i with (key[i] >> shift) >= c, for c in [0, nbins]; keys sorted
__global__ void k_build_ptr(const unsigned long long *__restrict__ k, int shift, int n, int nbins, int *ptr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    long long lo = (i == 0) ? 0 : (long long)(k[i - 1] >> shift) + 1;
    long long hi = (i == n) ? nbins : (long long)(k[i] >> shift);
    for (long long c = lo; c <= hi; c++) ptr[c] = i;
}
__global__ void k_low32(const unsigned long long *__restrict__ k, int *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)(k[i] & 0xffffffffULL);
}

// Two-pass segmented sums (setup): first[p] = the first entry of segment p; extra[p] = its
// remaining entry count; multi[p] = 1 when it has any.
__global__ void k_seg_first(const int *__restrict__ ptr, const int *__restrict__ perm, int n, int *first,
                            int *multi, int *extra) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int b = ptr[p], c = ptr[p + 1] - b;
    first[p] = c > 0 ? perm[b] : -1;
    multi[p] = c > 1;
    extra[p] = c > 1 ? c - 1 : 0;
}
// compacted multi-entry segments: mseg[i] = segment, mptr[i] = start of its extra entries in
// mperm (inclusive scans midx of multi and mcum of extra)
__global__ void k_seg_multi(const int *__restrict__ ptr, const int *__restrict__ perm, int n,
                            const int *__restrict__ multi, const int *__restrict__ midx,
                            const int *__restrict__ extra, const int *__restrict__ mcum, int *mseg, int *mptr,
                            int *mperm) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !multi[p]) return;
    const int i = midx[p] - 1, start = mcum[p] - extra[p];
    mseg[i] = p;
    mptr[i] = start;
    for (int j = 0; j < extra[p]; j++) mperm[start + j] = perm[ptr[p] + 1 + j];
}

// out[i] = arr[idx[i]] (setup)
__global__ void k_gather_i32(const int *__restrict__ arr, const long long *__restrict__ idx, int n, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = arr[idx[i]];
}
// out[i] = first position p in the ascending arr[0..n) with arr[p] >= key[i] (setup)
__global__ void k_lower_bound(const int *__restrict__ arr, int n, const long long *__restrict__ key, int nk,
                              int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        if ((long long)arr[mid] < key[i]) lo = mid + 1;
        else hi = mid;
    }
    out[i] = lo;
}

inline unsigned grid_of(i64 n, int b) { return (unsigned)((n + b - 1) / b); }

thread_local std::string g_create_err;

}  // namespace

// ------------------------------------------------------------------ the model
// A segmented sum over a sorted permutation (COO -> CSC, compressed Hessian -> CSC) in two passes:
// a gather of every segment's first entry (k_permute over first), then the remaining entries of
// the segments that have several, added onto the result in ascending order (k_seg_sum_warp<true>).
// The additions and their order are those of the one-pass sum, which starts from 0.0: the results
// are equal (bit for bit, except a one-entry segment holding -0.0, which the one-pass sum turns
// into +0.0).  Most CSC entries have one contributor, so most of the work is a plain permutation.
struct CscSum {
    int n = 0, n_multi = 0;
    int *first = nullptr, *mptr = nullptr, *mperm = nullptr, *mseg = nullptr;
};

struct exa_model {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = EXA_FP64;
    int block = 128;
    bool bounds_check = false;
    i64 nvar = 0, ncon = 0, npar = 0, nnzj = 0, nnzh = 0, nnzj_csc = 0, nnzh_csc = 0, nnzg = 0, naug = 0;
    int n_aug_rows = 0;
    int nb = 1;
    std::vector<i64> xoff, coff, joff, hoff;
    std::vector<exa::Pattern> pats;
    std::vector<exa::Group> groups;

    cudaLibrary_t lib = nullptr;
    cudaKernel_t fn[exa::M_COUNT] = {};
    int regs[exa::M_COUNT] = {};
    // fused step (EXA_FLAG_FUSED_STEP): kernels exa_step (index 0, tiles of M_ALL) and exa_step_b
    // (1, M_ALL_B), their work queues, per-member tile counts and the queue/tile counters
    bool fused_step = false;
    cudaKernel_t fn_step[2] = {};
    ExaTask *d_items[2] = {};
    int nitems[2] = {}, step_grid[2] = {};
    bool step_ready[2] = {};
    int *d_need[2] = {}, *d_sctr = nullptr;
    std::vector<ExaTile> h_tiles[exa::M_COUNT];  // host copies of the tile lists
    i64 objpart_n = 0;                           // objective partial slots allocated
    int step_hold = -1;  // failure injection: member whose tile count the next fused step cannot reach
    ExaPM *d_pm = nullptr;
    ExaTile *d_tiles[exa::M_COUNT] = {};
    int ntiles[exa::M_COUNT] = {};
    int grid[exa::M_COUNT] = {};  // CTAs launched per kernel kind (<= ntiles: persistent tile loop)
    int persist = 0;              // persistent grid factor chosen by the tuner (0: one CTA per tile)
    int min_blocks = 0;           // launch-bounds minimum CTAs per SM chosen by the tuner
    bool by_pattern = true;       // generated code emits each pattern's arithmetic next to its outputs
    int prefetch = 0;             // L2 prefetch depth of the generated tile loop (CodegenOptions)
    int lanes = 1;                // warp sets per instance of split groups (CodegenOptions)
    bool lazy_loads = false;      // with by_pattern: inputs loaded one pattern ahead (CodegenOptions)
    int stage = 0;                // inputs of the next tile staged in shared memory (CodegenOptions)
    int dsmem[exa::M_COUNT] = {}; // dynamic shared memory of each kernel kind (bytes)
    int wave_pct = 0;             // persistent evaluation grid of this % of one wave (0: off)
    int pfd[exa::M_COUNT] = {};   // prefetch distance in tiles per kernel kind (0: none)
    bool split_all = false;       // exa_eval_all: first- and second-order kernels instead of one
    bool csc_direct = false;      // duplicate-free CSC written by the evaluation kernel (scatter)
    std::vector<ExaPM> h_pms;     // host copy of the group descriptors
    // CUDA graphs of exa_eval_all, one per argument tuple
    struct GraphEntry {
        std::array<const void *, 10> key;
        cudaGraphExec_t exec;
        uint64_t last_use;
    };
    std::vector<GraphEntry> graphs;
    uint64_t graph_clock = 0;
    int graph_kernels = 0;  // kernel launches in the most recently captured exa_eval_all graph
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;
    // exa_eval_all runs its independent reductions on side streams forked from and joined back into
    // the model stream: 0 the Jacobian CSC (and member chunks' reductions), 1 the Hessian CSC, 3 the
    // split mode's first-order sums (2 is not used)
    cudaStream_t side[4] = {};
    // device buffers of exa_eval_all_host: x, y, f, g, c, jac, hess, jac_csc, hess_csc
    double *d_host_io[9] = {};
    cudaEvent_t ev_fork = nullptr, ev_first = nullptr, ev_join[4] = {};
    double *d_theta = nullptr;
    int *d_status = nullptr;
    int *d_jrow = nullptr, *d_jcol = nullptr, *d_hrow = nullptr, *d_hcol = nullptr, *d_gvar = nullptr, *d_arow = nullptr;
    // Jacobian: CSC (segments over the (col,row)-sorted COO) and row grouping
    int *d_jperm = nullptr, *d_jsegptr = nullptr, *d_jcolptr = nullptr, *d_jrowval = nullptr, *d_jcoo2csc = nullptr;
    int *d_jcolptr_coo = nullptr, *d_jrperm = nullptr, *d_jrptr = nullptr;
    // Hessian: same
    int *d_hperm = nullptr, *d_hsegptr = nullptr, *d_hcolptr = nullptr, *d_hrowval = nullptr, *d_hcoo2csc = nullptr;
    // compressed Hessian (per-instance sums of a group's slots with equal (row, col)): structure,
    // permutation sorted by (col, row) and segment pointers per Hessian CSC entry
    i64 nnzhc = 0;
    bool has_hcomp = false;       // group-compressed Hessian sums exist (fewer than the COO slots)
    // sparse gradient: zero fill plus sums over the variables that have gradient slots only
    CscSum sum_j, sum_h, sum_hc;  // Jacobian CSC (when it has duplicates), Hessian CSC, from compressed sums
    // Member-chunked exa_eval_all: the members are split into nchunks contiguous groups; the
    // evaluation of group c + 1 runs on the model stream while the reductions of group c run on a
    // side stream.  Per member b (nb + 1 boundaries each): first tile of every kernel kind, and the
    // first position of b's part of every reduction's output or work list.
    int nchunks = 1;
    bool chunks_fixed = false;  // given at creation: the tuner keeps it
    bool wave_fixed = false;    // wave_pct given at creation: the tuner keeps it
    std::vector<int> chunk_b;  // member boundaries of the chunks (nchunks + 1)
    std::vector<int> mb_tile[exa::M_COUNT];
    std::vector<int> mb_jcsc, mb_hcsc, mb_jmulti, mb_hmulti, mb_hcmulti, mb_gseg, mb_arow;
    cudaEvent_t ev_chunk[16] = {};
    // Hooks of eval_all_chunked, called before chunk k's evaluation is enqueued and after its
    // reductions are (the host-buffer pipeline of exa_eval_all_host); empty otherwise.
    std::function<exa_status(int)> pre_chunk, post_chunk;
    // exa_eval_all_host pipeline: copy streams and per-chunk events (inputs in, outputs final)
    bool host_serial = false;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[16] = {}, ev_out[16] = {}, ev_hstart = nullptr, ev_hdone = nullptr;
    // timing events around the evaluation kernel(s) of the latest exa_eval_all step (recorded into
    // the cached graphs too); exa_stat "eval_kernel_ms" reads them
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
    bool ev_k_valid = false;
    bool grad_compact = false;
    int n_gseg = 0;
    int *d_gsegptr = nullptr, *d_gsegvar = nullptr;
    bool use_hcomp = false;       // ... and feed the Hessian CSC (tuner choice)
    int *d_hcrow = nullptr, *d_hccol = nullptr, *d_hcperm = nullptr, *d_hcsegptr = nullptr;
    double *d_hcbuf = nullptr;
    // Hessian CSC seen by rows (products): column of each CSC entry, row-sorted permutation
    int *d_hcolof = nullptr, *d_hcsr_perm = nullptr, *d_hcsr_ptr = nullptr;
    double *d_hcscbuf = nullptr;
    // gradient and augmentation segments
    int *d_gperm = nullptr, *d_gptr = nullptr;
    int *d_aperm = nullptr, *d_aptr = nullptr, *d_arows = nullptr;
    // work buffers
    double *d_jbuf = nullptr, *d_hbuf = nullptr, *d_gbuf = nullptr, *d_abuf = nullptr, *d_objpart = nullptr,
           *d_cbuf = nullptr;
    std::vector<void *> allocs;
    size_t device_bytes = 0;
    double nvrtc_ms = 0, create_ms = 0, tune_ms = 0;
    std::string err;
};

extern "C" {
static exa_status eval_all_launches(exa_model *m, const double *x, const double *y, double sigma, double *f,
                                    double *g, double *c, double *jac, double *hess, double *jac_csc,
                                    double *hess_csc);
static exa_status prepare_step(exa_model *m);
}

namespace {

exa_status fail(exa_model *m, exa_status s, const std::string &msg) {
    if (m) m->err = msg;
    return s;
}

template <typename T>
cudaError_t dalloc(exa_model *m, T **p, i64 count) {
    *p = nullptr;
    size_t bytes = (size_t)std::max<i64>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) {
        m->allocs.push_back(*p);
        m->device_bytes += bytes;
    }
    return e;
}

#define CR(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(m, e_ == cudaErrorMemoryAllocation ? EXA_E_OOM : EXA_E_CUDA,               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

void free_all(exa_model *m) {
    for (auto &ge : m->graphs) cudaGraphExecDestroy(ge.exec);
    m->graphs.clear();
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    m->cap_stream = nullptr;
    for (int s = 0; s < 4; s++) {
        if (m->side[s]) cudaStreamDestroy(m->side[s]);
        if (m->ev_join[s]) cudaEventDestroy(m->ev_join[s]);
        m->side[s] = nullptr;
        m->ev_join[s] = nullptr;
    }
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_first) cudaEventDestroy(m->ev_first);
    m->ev_fork = nullptr;
    m->ev_first = nullptr;
    for (cudaEvent_t &e : m->ev_chunk) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    for (cudaEvent_t *e : {&m->ev_hstart, &m->ev_hdone, &m->ev_k0, &m->ev_k1}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    m->ev_k_valid = false;
    for (int k = 0; k < 16; k++)
        for (cudaEvent_t *e : {&m->ev_in[k], &m->ev_out[k]}) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
    for (cudaStream_t *st : {&m->h2d, &m->d2h}) {
        if (*st) cudaStreamDestroy(*st);
        *st = nullptr;
    }
    for (int i = 0; i < 2; i++) {
        if (m->d_items[i]) cudaFree(m->d_items[i]);
        if (m->d_need[i]) cudaFree(m->d_need[i]);
        m->d_items[i] = nullptr;
        m->d_need[i] = nullptr;
        m->step_ready[i] = false;
    }
    if (m->d_sctr) cudaFree(m->d_sctr);
    m->d_sctr = nullptr;
    for (int k = 0; k < exa::M_COUNT; k++) {
        if (m->d_tiles[k]) cudaFree(m->d_tiles[k]);
        m->d_tiles[k] = nullptr;
    }
    for (void *p : m->allocs) cudaFree(p);
    m->allocs.clear();
    if (m->lib) cudaLibraryUnload(m->lib);
    m->lib = nullptr;
}

exa_status nvrtc_compile(exa_model *m, const std::string &src, std::vector<char> &cubin) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "exa_generated.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return fail(m, EXA_E_NVRTC, "nvrtcCreateProgram failed");
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "--fmad=true",
                          "-default-device"};
    nvrtcResult r = nvrtcCompileProgram(prog, sizeof(opts) / sizeof(opts[0]), opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        return fail(m, EXA_E_NVRTC, std::string("NVRTC: ") + nvrtcGetErrorString(r) + "\n" + log.substr(0, 4000));
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin.resize(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    return EXA_OK;
}

// Process-wide cache of compiled modules keyed by the generated source: models that share their
// pattern trees and options (batch members, or the same model created twice) compile once.
std::mutex g_cubin_mu;
std::map<std::string, std::shared_ptr<std::vector<char>>> g_cubins;

// Compiles the kernels of several code-generator variants into the module cache at once, one
// thread per variant (NVRTC is thread-safe): the tuner then loads each variant from the cache.
// Failures are left for the variant's own compile to report.
void precompile(const exa_model *m, const std::vector<exa::CodegenOptions> &variants) {
    std::vector<std::string> srcs;
    for (const exa::CodegenOptions &cg : variants) {
        std::string gerr;
        std::string src = exa::generate_source(m->pats, m->groups, cg, &gerr);
        if (!gerr.empty()) continue;
        std::lock_guard<std::mutex> lk(g_cubin_mu);
        if (!g_cubins.count(src)) srcs.push_back(std::move(src));
    }
    std::vector<std::thread> th;
    for (const std::string &src : srcs)
        th.emplace_back([&src]() {
            exa_model scratch;
            auto cubin = std::make_shared<std::vector<char>>();
            if (nvrtc_compile(&scratch, src, *cubin) != EXA_OK) return;
            std::lock_guard<std::mutex> lk(g_cubin_mu);
            if (g_cubins.size() > 64) g_cubins.clear();
            g_cubins[src] = cubin;
        });
    for (std::thread &t : th) t.join();
}

exa_status compile(exa_model *m, const std::string &src) {
    auto t0 = std::chrono::steady_clock::now();
    std::shared_ptr<std::vector<char>> cubin;
    {
        std::lock_guard<std::mutex> lk(g_cubin_mu);
        auto it = g_cubins.find(src);
        if (it != g_cubins.end()) cubin = it->second;
    }
    if (!cubin) {
        cubin = std::make_shared<std::vector<char>>();
        if (exa_status e = nvrtc_compile(m, src, *cubin)) return e;
        std::lock_guard<std::mutex> lk(g_cubin_mu);
        if (g_cubins.size() > 64) g_cubins.clear();
        g_cubins[src] = cubin;
    }
    m->nvrtc_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    CR(cudaLibraryLoadData(&m->lib, cubin->data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    for (int k = 0; k < exa::M_COUNT; k++) {
        std::string name = std::string("exa_") + exa::kModeName[k];
        CR(cudaLibraryGetKernel(&m->fn[k], m->lib, name.c_str()));
        if (m->dsmem[k] > 0)
            CR(cudaFuncSetAttribute((const void *)m->fn[k], cudaFuncAttributeMaxDynamicSharedMemorySize, m->dsmem[k]));
        cudaFuncAttributes attr;
        CR(cudaFuncGetAttributes(&attr, (const void *)m->fn[k]));
        m->regs[k] = attr.numRegs;
    }
    for (int i = 0; i < 2; i++) {  // present only when generated with the fused step
        m->fn_step[i] = nullptr;
        m->step_ready[i] = false;
        if (!m->fused_step) continue;
        CR(cudaLibraryGetKernel(&m->fn_step[i], m->lib, i ? "exa_step_b" : "exa_step"));
    }
    return EXA_OK;
}

// The evaluation kernel of `mode` over its tiles [t0, t1) (t1 < 0: all tiles) on stream st (null:
// the model stream).
// CTAs of one launch of kernel kind `mode` over nt tiles; kinds that reduce objective terms write one
// partial sum per CTA.
int eval_grid(const exa_model *m, Mode mode, int nt) { return m->grid[mode] > 0 ? std::min(m->grid[mode], nt) : nt; }

exa_status launch_eval(exa_model *m, Mode mode, const double *x, const double *y, double sigma, ExaOut out,
                       int t0 = 0, int t1 = -1, cudaStream_t st = nullptr) {
    if (t1 < 0) t1 = m->ntiles[mode];
    if (t1 <= t0) return EXA_OK;
    out.status = m->d_status;
    ExaStructOut so{};
    so.status = m->d_status;
    const double *th = m->d_theta;
    int nt = t1 - t0;
    const ExaTile *tiles = m->d_tiles[mode] + t0;
    int pfd = m->pfd[mode];
    void *args[] = {&tiles, &nt, &m->d_pm, &x, &y, &th, &sigma, &out, &so, &pfd};
    const int grid = eval_grid(m, mode, nt);
    CR(cudaLaunchKernel((const void *)m->fn[mode], dim3(grid), dim3(m->block), args, (size_t)m->dsmem[mode],
                        st ? st : m->stream));
    return EXA_OK;
}

exa_status check_model(exa_model *m) {
    if (!m) return EXA_E_INVALID;
    CR(cudaSetDevice(m->device));
    return EXA_OK;
}

// Sorted-key helpers used by the structure setup -----------------------------------------------
struct Scratch {
    exa_model *m;
    std::vector<void *> mine;
    ~Scratch() {
        for (void *p : mine) cudaFree(p);
    }
    template <typename T>
    cudaError_t get(T **p, i64 n) {
        cudaError_t e = cudaMalloc((void **)p, (size_t)std::max<i64>(n, 1) * sizeof(T));
        if (e == cudaSuccess) mine.push_back(*p);
        return e;
    }
};

// Sort keys with values 0..n-1 (stable): sorted keys and permutation.
exa_status sort_with_perm(exa_model *m, Scratch &S, unsigned long long *keys, int n, int end_bit,
                          unsigned long long **skeys, int *perm) {
    int *iota = nullptr;
    CR(S.get(&iota, n));
    CR(S.get(skeys, n));
    if (n > 0) {
        k_iota<<<grid_of(n, 256), 256, 0, m->stream>>>(iota, n);
        CR(cudaGetLastError());
        CR(exa_sort_pairs_u64(keys, *skeys, iota, perm, n, end_bit, m->stream));
    }
    return EXA_OK;
}

// Segments of equal sorted keys: count, start positions, keys, and (optional) position -> segment.
exa_status segments(exa_model *m, Scratch &S, const unsigned long long *skeys, const int *perm, int n,
                    int *nseg, int **segptr, unsigned long long **segkey, int *coo2seg, bool persistent_ptr) {
    int *flag = nullptr, *segid = nullptr;
    CR(S.get(&flag, n));
    CR(S.get(&segid, n));
    *nseg = 0;
    if (n > 0) {
        k_new_segment<<<grid_of(n, 256), 256, 0, m->stream>>>(skeys, flag, n);
        CR(cudaGetLastError());
        CR(exa_inclusive_sum_i32(flag, segid, n, m->stream));
        CR(cudaMemcpy(nseg, segid + n - 1, sizeof(int), cudaMemcpyDeviceToHost));
    }
    if (persistent_ptr) CR(dalloc(m, segptr, (i64)*nseg + 1));
    else CR(S.get(segptr, (i64)*nseg + 1));
    CR(S.get(segkey, *nseg));
    if (n > 0) {
        k_segments<<<grid_of(n, 256), 256, 0, m->stream>>>(skeys, flag, segid, perm, *segptr, *segkey, coo2seg, n);
        CR(cudaGetLastError());
    } else {
        CR(cudaMemset(*segptr, 0, sizeof(int)));
    }
    return EXA_OK;
}

exa_status build_ptr(exa_model *m, const unsigned long long *skeys, int shift, int n, i64 nbins, int **ptr) {
    CR(dalloc(m, ptr, nbins + 1));
    k_build_ptr<<<grid_of((i64)n + 1, 256), 256, 0, m->stream>>>(skeys, shift, n, (int)nbins, *ptr);
    CR(cudaGetLastError());
    return EXA_OK;
}

exa_status build_csc_sum(exa_model *m, Scratch &S, const int *ptr, const int *perm, int n, CscSum *cs) {
    cs->n = n;
    CR(dalloc(m, &cs->first, n));
    if (n <= 0) return EXA_OK;
    int *multi = nullptr, *extra = nullptr, *midx = nullptr, *mcum = nullptr;
    CR(S.get(&multi, n));
    CR(S.get(&extra, n));
    CR(S.get(&midx, n));
    CR(S.get(&mcum, n));
    k_seg_first<<<grid_of(n, 256), 256, 0, m->stream>>>(ptr, perm, n, cs->first, multi, extra);
    CR(cudaGetLastError());
    CR(exa_inclusive_sum_i32(multi, midx, n, m->stream));
    CR(exa_inclusive_sum_i32(extra, mcum, n, m->stream));
    int nm = 0, ne = 0;
    CR(cudaMemcpyAsync(&nm, midx + n - 1, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CR(cudaMemcpyAsync(&ne, mcum + n - 1, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CR(cudaStreamSynchronize(m->stream));
    cs->n_multi = nm;
    CR(dalloc(m, &cs->mseg, nm));
    CR(dalloc(m, &cs->mptr, (i64)nm + 1));
    CR(dalloc(m, &cs->mperm, ne));
    k_seg_multi<<<grid_of(n, 256), 256, 0, m->stream>>>(ptr, perm, n, multi, midx, extra, mcum, cs->mseg, cs->mptr,
                                                         cs->mperm);
    CR(cudaGetLastError());
    CR(cudaMemcpyAsync(cs->mptr + nm, &ne, sizeof(int), cudaMemcpyHostToDevice, m->stream));
    CR(cudaStreamSynchronize(m->stream));
    return EXA_OK;
}

// Per-member boundaries of every reduction's output and work lists (for member-chunked evaluation).
exa_status build_member_bounds(exa_model *m) {
    Scratch S{m};
    const int nb = m->nb;
    long long *key = nullptr;
    int *out = nullptr;
    CR(S.get(&key, nb + 1));
    CR(S.get(&out, nb + 1));
    std::vector<long long> k(nb + 1);
    auto fetch = [&](std::vector<int> &dst) -> exa_status {
        dst.assign(nb + 1, 0);
        CR(cudaMemcpy(dst.data(), out, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost));
        return EXA_OK;
    };
    auto gather = [&](const int *arr, const std::vector<i64> &idx, std::vector<int> &dst) -> exa_status {
        for (int b = 0; b <= nb; b++) k[b] = idx[b];
        CR(cudaMemcpy(key, k.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice));
        k_gather_i32<<<grid_of(nb + 1, 256), 256, 0, m->stream>>>(arr, key, nb + 1, out);
        CR(cudaGetLastError());
        return fetch(dst);
    };
    auto lower = [&](const int *arr, int n, const std::vector<long long> &keys, std::vector<int> &dst) -> exa_status {
        CR(cudaMemcpy(key, keys.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice));
        k_lower_bound<<<grid_of(nb + 1, 256), 256, 0, m->stream>>>(arr, n, key, nb + 1, out);
        CR(cudaGetLastError());
        return fetch(dst);
    };
    auto as_ll = [&](const std::vector<int> &v) { return std::vector<long long>(v.begin(), v.end()); };
    if (exa_status e = gather(m->d_jcolptr, m->xoff, m->mb_jcsc)) return e;
    if (exa_status e = gather(m->d_hcolptr, m->xoff, m->mb_hcsc)) return e;
    m->mb_jmulti.assign(nb + 1, 0);
    m->mb_hmulti.assign(nb + 1, 0);
    m->mb_hcmulti.assign(nb + 1, 0);
    if (m->sum_j.n_multi)
        if (exa_status e = lower(m->sum_j.mseg, m->sum_j.n_multi, as_ll(m->mb_jcsc), m->mb_jmulti)) return e;
    if (m->sum_h.n_multi)
        if (exa_status e = lower(m->sum_h.mseg, m->sum_h.n_multi, as_ll(m->mb_hcsc), m->mb_hmulti)) return e;
    if (m->sum_hc.n_multi)
        if (exa_status e = lower(m->sum_hc.mseg, m->sum_hc.n_multi, as_ll(m->mb_hcsc), m->mb_hcmulti)) return e;
    m->mb_gseg.assign(nb + 1, 0);
    if (m->n_gseg)
        if (exa_status e = lower(m->d_gsegvar, m->n_gseg, std::vector<long long>(m->xoff.begin(), m->xoff.end()),
                                 m->mb_gseg)) return e;
    m->mb_arow.assign(nb + 1, 0);
    if (m->n_aug_rows)
        if (exa_status e = lower(m->d_arows, m->n_aug_rows, std::vector<long long>(m->coff.begin(), m->coff.end()),
                                 m->mb_arow)) return e;
    return EXA_OK;
}

// Member boundaries of n chunks of about equal nonzeros (n = 1: one chunk of all members).
void set_chunks(exa_model *m, int n) {
    const int nb = m->nb;
    n = std::max(1, std::min(n, std::min(nb, 16)));
    m->nchunks = n;
    m->chunk_b.assign(1, 0);
    const double tot = (double)(m->nnzj + m->nnzh);
    for (int c = 1; c < n; c++) {
        int b = m->chunk_b.back() + 1;
        while (b < nb && (double)(m->joff[b] + m->hoff[b]) < tot * c / n) b++;
        m->chunk_b.push_back(std::min(b, nb - (n - c)));
    }
    m->chunk_b.push_back(nb);
}

// Per-model structure: CSC of J and H, row groupings, gradient and augmentation segments.
exa_status build_structure(exa_model *m) {
    Scratch S{m};
    const int nj = (int)m->nnzj, nh = (int)m->nnzh, ng = (int)m->nnzg, na = (int)m->naug;
    unsigned long long *keys = nullptr, *skeys = nullptr, *segkey = nullptr;
    int nseg = 0;
    // ---- Jacobian CSC: sort (col, row)
    CR(S.get(&keys, std::max({nj, nh, ng, na, 1})));
    CR(dalloc(m, &m->d_jperm, nj));
    CR(dalloc(m, &m->d_jcoo2csc, nj));
    if (nj) {
        k_keys2<<<grid_of(nj, 256), 256, 0, m->stream>>>(m->d_jcol, m->d_jrow, keys, nj);
        CR(cudaGetLastError());
    }
    if (exa_status e = sort_with_perm(m, S, keys, nj, 64, &skeys, m->d_jperm)) return e;
    if (exa_status e = segments(m, S, skeys, m->d_jperm, nj, &nseg, &m->d_jsegptr, &segkey, m->d_jcoo2csc, true)) return e;
    m->nnzj_csc = nseg;
    if (nseg < nj)
        if (exa_status e = build_csc_sum(m, S, m->d_jsegptr, m->d_jperm, nseg, &m->sum_j)) return e;
    CR(dalloc(m, &m->d_jrowval, nseg));
    if (nseg) {
        k_low32<<<grid_of(nseg, 256), 256, 0, m->stream>>>(segkey, m->d_jrowval, nseg);
        CR(cudaGetLastError());
    }
    if (exa_status e = build_ptr(m, segkey, 32, nseg, m->nvar, &m->d_jcolptr)) return e;
    if (exa_status e = build_ptr(m, skeys, 32, nj, m->nvar, &m->d_jcolptr_coo)) return e;
    // ---- Jacobian row grouping
    CR(dalloc(m, &m->d_jrperm, nj));
    if (nj) {
        k_keys1<<<grid_of(nj, 256), 256, 0, m->stream>>>(m->d_jrow, keys, nj);
        CR(cudaGetLastError());
    }
    if (exa_status e = sort_with_perm(m, S, keys, nj, 32, &skeys, m->d_jrperm)) return e;
    if (exa_status e = build_ptr(m, skeys, 0, nj, m->ncon, &m->d_jrptr)) return e;

    // ---- Hessian CSC
    CR(dalloc(m, &m->d_hperm, nh));
    CR(dalloc(m, &m->d_hcoo2csc, nh));
    if (nh) {
        k_keys2<<<grid_of(nh, 256), 256, 0, m->stream>>>(m->d_hcol, m->d_hrow, keys, nh);
        CR(cudaGetLastError());
    }
    if (exa_status e = sort_with_perm(m, S, keys, nh, 64, &skeys, m->d_hperm)) return e;
    if (exa_status e = segments(m, S, skeys, m->d_hperm, nh, &nseg, &m->d_hsegptr, &segkey, m->d_hcoo2csc, true)) return e;
    m->nnzh_csc = nseg;
    if (nseg < nh)
        if (exa_status e = build_csc_sum(m, S, m->d_hsegptr, m->d_hperm, nseg, &m->sum_h)) return e;
    CR(dalloc(m, &m->d_hrowval, nseg));
    if (nseg) {
        k_low32<<<grid_of(nseg, 256), 256, 0, m->stream>>>(segkey, m->d_hrowval, nseg);
        CR(cudaGetLastError());
    }
    if (exa_status e = build_ptr(m, segkey, 32, nseg, m->nvar, &m->d_hcolptr)) return e;

    // ---- compressed Hessian: its (col, row)-sorted segments are the Hessian CSC entries
    if (m->has_hcomp) {
        const int nc = (int)m->nnzhc;
        unsigned long long *ck = nullptr;
        CR(S.get(&ck, nc));
        CR(dalloc(m, &m->d_hcperm, nc));
        k_keys2<<<grid_of(nc, 256), 256, 0, m->stream>>>(m->d_hccol, m->d_hcrow, ck, nc);
        CR(cudaGetLastError());
        if (exa_status e = sort_with_perm(m, S, ck, nc, 64, &skeys, m->d_hcperm)) return e;
        int nsc = 0;
        if (exa_status e = segments(m, S, skeys, m->d_hcperm, nc, &nsc, &m->d_hcsegptr, &segkey, nullptr, true)) return e;
        if (nsc != m->nnzh_csc) return fail(m, EXA_E_INTERNAL, "compressed Hessian does not cover the CSC entries");
        if (exa_status e = build_csc_sum(m, S, m->d_hcsegptr, m->d_hcperm, nsc, &m->sum_hc)) return e;
        CR(dalloc(m, &m->d_hcbuf, nc));
    }

    // ---- Hessian CSC by rows (for products)
    {
        const int nc = (int)m->nnzh_csc;
        CR(dalloc(m, &m->d_hcolof, nc));
        CR(dalloc(m, &m->d_hcsr_perm, nc));
        CR(dalloc(m, &m->d_hcscbuf, nc));
        if (m->nvar) {
            k_col_of<<<grid_of(m->nvar, 256), 256, 0, m->stream>>>(m->d_hcolptr, m->d_hcolof, (int)m->nvar);
            CR(cudaGetLastError());
        }
        if (nc) {
            k_keys2<<<grid_of(nc, 256), 256, 0, m->stream>>>(m->d_hrowval, m->d_hcolof, keys, nc);
            CR(cudaGetLastError());
        }
        if (exa_status e = sort_with_perm(m, S, keys, nc, 64, &skeys, m->d_hcsr_perm)) return e;
        if (exa_status e = build_ptr(m, skeys, 32, nc, m->nvar, &m->d_hcsr_ptr)) return e;
    }

    // ---- gradient segments by variable
    CR(dalloc(m, &m->d_gperm, ng));
    if (ng) {
        k_keys1<<<grid_of(ng, 256), 256, 0, m->stream>>>(m->d_gvar, keys, ng);
        CR(cudaGetLastError());
    }
    if (exa_status e = sort_with_perm(m, S, keys, ng, 32, &skeys, m->d_gperm)) return e;
    if (exa_status e = build_ptr(m, skeys, 0, ng, m->nvar, &m->d_gptr)) return e;
    // the variables that have gradient slots, for the compact form (chosen when they are fewer than
    // half of the variables)
    if (exa_status e = segments(m, S, skeys, m->d_gperm, ng, &nseg, &m->d_gsegptr, &segkey, nullptr, true)) return e;
    m->n_gseg = nseg;
    CR(dalloc(m, &m->d_gsegvar, nseg));
    if (nseg) {
        k_low32<<<grid_of(nseg, 256), 256, 0, m->stream>>>(segkey, m->d_gsegvar, nseg);
        CR(cudaGetLastError());
    }
    m->grad_compact = 2 * (i64)nseg < m->nvar;

    // ---- augmentation segments by row (only rows that receive terms)
    CR(dalloc(m, &m->d_aperm, na));
    if (na) {
        k_keys1<<<grid_of(na, 256), 256, 0, m->stream>>>(m->d_arow, keys, na);
        CR(cudaGetLastError());
    }
    if (exa_status e = sort_with_perm(m, S, keys, na, 32, &skeys, m->d_aperm)) return e;
    if (exa_status e = segments(m, S, skeys, m->d_aperm, na, &nseg, &m->d_aptr, &segkey, nullptr, true)) return e;
    m->n_aug_rows = nseg;
    CR(dalloc(m, &m->d_arows, nseg));
    if (nseg) {
        k_low32<<<grid_of(nseg, 256), 256, 0, m->stream>>>(segkey, m->d_arows, nseg);
        CR(cudaGetLastError());
    }
    CR(cudaStreamSynchronize(m->stream));
    return EXA_OK;
}

// Same tree shape: identical nodes except for the values of constants (index constants and
// value constants may differ between batch members; they become per-member descriptor values).
bool same_shape(const exa_pattern_desc &a, const exa_pattern_desc &b) {
    if (a.kind != b.kind || a.n_vnodes != b.n_vnodes || a.n_inodes != b.n_inodes || a.n_fields != b.n_fields ||
        a.row_root != b.row_root)
        return false;
    for (int i = 0; i < a.n_vnodes; i++) {
        const exa_vnode &u = a.vnodes[i], &v = b.vnodes[i];
        if (u.op != v.op || u.a != v.a || u.b != v.b) return false;
        if (u.op != EXA_V_CONST && u.ival != v.ival) return false;
    }
    for (int i = 0; i < a.n_inodes; i++) {
        const exa_inode &u = a.inodes[i], &v = b.inodes[i];
        if (u.op != v.op || u.a != v.a || u.b != v.b) return false;
        if (u.op != EXA_I_CONST && u.ival != v.ival) return false;
    }
    for (int f = 0; f < a.n_fields; f++)
        if (a.fields[f].type != b.fields[f].type) return false;
    return true;
}

exa_status load_patterns(const exa_model_desc &d0, exa_model *m) {
    const int np = d0.n_patterns;
    m->pats.resize(np);
    for (int p = 0; p < np; p++) {
        const exa_pattern_desc &pd = d0.patterns[p];
        exa::Pattern &P = m->pats[p];
        P.kind = pd.kind;
        P.n_inst = pd.n_inst;
        P.row_base = pd.row_base;
        P.row_limit = pd.row_limit;
        P.row_root = pd.row_root;
        for (int i = 0; i < pd.n_vnodes; i++) {
            const exa_vnode &v = pd.vnodes[i];
            P.v.push_back({v.op, v.a, v.b, v.ival, v.fval});
        }
        for (int i = 0; i < pd.n_inodes; i++) {
            const exa_inode &v = pd.inodes[i];
            P.ix.push_back({v.op, v.a, v.b, v.ival});
        }
        for (int f = 0; f < pd.n_fields; f++) P.ftype.push_back(pd.fields[f].type);
        std::string e = exa::analyse_pattern(P);
        if (!e.empty()) return fail(m, EXA_E_INVALID, "pattern " + std::to_string(p) + ": " + e);
    }
    return EXA_OK;
}

// Generates, compiles and loads the kernels for `block` threads per CTA and rebuilds the tile lists
// (member-major, then groups in declaration order; BLOCK instances per tile).
exa_status setup_kernels(exa_model *m, int block, int min_blocks = 0) {
    m->block = block;
    m->min_blocks = min_blocks;
    exa::CodegenOptions cg;
    cg.precision = m->precision;
    cg.block = block;
    cg.min_blocks = min_blocks;
    cg.bounds_check = m->bounds_check;
    cg.by_pattern = m->by_pattern;
    cg.prefetch = m->lanes > 1 ? 0 : m->prefetch;
    cg.lanes = m->lanes;
    cg.lazy_loads = m->lazy_loads;
    cg.stage = m->fused_step ? 0 : m->stage;
    cg.fused_step = m->fused_step;
    std::string gerr;
    std::string src = exa::generate_source(m->pats, m->groups, cg, &gerr, m->dsmem);
    if (!gerr.empty()) return fail(m, EXA_E_INTERNAL, gerr);
    if (getenv("EXA_DUMP_SOURCE")) {
        FILE *fp = fopen(getenv("EXA_DUMP_SOURCE"), "w");
        if (fp) { fputs(src.c_str(), fp); fclose(fp); }
    }
    if (m->lib) {
        cudaLibraryUnload(m->lib);
        m->lib = nullptr;
    }
    if (exa_status e = compile(m, src)) return e;
    const int ng = (int)m->groups.size(), nb = m->nb;
    for (int k = 0; k < exa::M_COUNT; k++) {
        std::vector<ExaTile> tiles;
        m->mb_tile[k].assign(nb + 1, 0);
        for (int b = 0; b < nb; b++)
            for (int gi = 0; gi < ng; gi++) {
                if (gi == 0) m->mb_tile[k][b] = (int)tiles.size();
                bool in = false;
                for (int p : m->groups[gi].pats) in = in || exa::pattern_in_mode(m->pats[p], (exa::Mode)k);
                if (!in) continue;
                const ExaPM &pm = m->h_pms[(size_t)b * ng + gi];
                // a group split into warp sets takes block / sets instances per tile
                const int per = block / (int)exa::group_sets(m->pats, m->groups[gi], (exa::Mode)k, m->lanes).size();
                for (i64 s = 0; s < pm.n_inst; s += per)
                    tiles.push_back({b * ng + gi, (int)s});
            }
        m->ntiles[k] = (int)tiles.size();
        m->mb_tile[k][nb] = m->ntiles[k];
        m->h_tiles[k] = tiles;
        m->grid[k] = m->ntiles[k];
        m->pfd[k] = 0;
        if (m->d_tiles[k]) cudaFree(m->d_tiles[k]);
        m->d_tiles[k] = nullptr;
        m->step_ready[0] = m->step_ready[1] = false;  // the fused step's queues index these tiles
        CR(cudaMalloc((void **)&m->d_tiles[k], sizeof(ExaTile) * std::max<size_t>(tiles.size(), 1)));
        if (!tiles.empty())
            CR(cudaMemcpy(m->d_tiles[k], tiles.data(), sizeof(ExaTile) * tiles.size(), cudaMemcpyHostToDevice));
    }
    return EXA_OK;
}

// Persistent grid for every kernel kind: factor x resident CTAs per SM x SMs (0: one CTA per tile).
// Prefetch distance: a CTA's next tile in a persistent grid; with one CTA per tile, the tile that
// starts about one wave of resident CTAs later.
exa_status apply_grid(exa_model *m, int factor) {
    m->persist = factor;
    int sms = 0;
    CR(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    for (int k = 0; k < exa::M_COUNT; k++) {
        m->grid[k] = m->ntiles[k];
        m->pfd[k] = 0;
        if (k == exa::M_STRUCT) continue;
        int occ = 0;
        CR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)m->fn[k], m->block, (size_t)m->dsmem[k]));
        const long long wave = (long long)std::max(occ, 1) * sms;
        const long long g = (long long)std::max(factor, 0) * wave;
        if (factor > 0 && g < m->ntiles[k]) m->grid[k] = (int)g;
        if (m->wave_pct > 0) {  // less than one wave: room on every SM for work on other streams
            const long long gp = std::max<long long>(1, (wave * m->wave_pct + 99) / 100);
            if (gp < m->ntiles[k]) m->grid[k] = (int)gp;
        }
        if (m->prefetch > 0) m->pfd[k] = (int)std::min<long long>(m->grid[k] < m->ntiles[k] ? m->grid[k] : wave, 1 << 30);
    }
    return EXA_OK;
}

// Launch-shape autotuner, in stages, each keeping the fastest variant: (1) the fused evaluation
// kernel (everything, at varied inputs of unit size) for 64 / 128 / 256 threads per CTA and one CTA
// per tile versus persistent grids of 1, 2 and 4 waves of resident CTAs; (2) for that shape, launch
// bounds for 20 to 32 resident warps per SM or none, with each of the three emission orders of the
// generated arithmetic; (3) L2 prefetch depth; (4) two warp sets per instance; (5) shared-memory
// staging of the next tile's inputs, with its own register cap and grid search; (6) whole
// exa_eval_all steps with every output: member chunks and partial waves, compressed or COO
// Hessian sums for the CSC, fused or split first/second order, CSC gathered or scattered.  The
// code-generator variants of a stage are compiled in parallel before they are timed.  Models too
// small to fill the GPU are not tuned.
exa_status autotune(exa_model *m) {
    int sms = 0;
    CR(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    if (m->ntiles[exa::M_ALL] < 4 * sms) return EXA_OK;
    Scratch S{m};
    double *x = nullptr, *y = nullptr, *part = nullptr;
    CR(S.get(&x, m->nvar));
    CR(S.get(&y, m->ncon));
    // tuning inputs: deterministic, varied and of unit size (x in [0.9, 1.1], y in [-1, 1], from
    // golden-ratio sequences), so that angle differences, products and derivatives are nonzero
    // as at a real iterate (constant inputs would make many of them exactly zero, which takes other
    // branches in the exact conversions of the mixed mode)
    std::vector<double> hv((size_t)std::max<i64>(std::max(m->nvar, m->ncon), 1));
    for (size_t i = 0; i < hv.size(); i++) hv[i] = 0.9 + 0.2 * std::fmod(0.6180339887498949 * (double)(i + 1), 1.0);
    CR(cudaMemcpy(x, hv.data(), sizeof(double) * m->nvar, cudaMemcpyHostToDevice));
    for (size_t i = 0; i < hv.size(); i++) hv[i] = -1.0 + 2.0 * std::fmod(0.7548776662466927 * (double)(i + 1), 1.0);
    if (m->ncon) CR(cudaMemcpy(y, hv.data(), sizeof(double) * m->ncon, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CR(cudaEventCreate(&e0));
    CR(cudaEventCreate(&e1));
    // one warm call, then the best of three rounds of `reps` calls (milliseconds per round): the
    // rounds make the choice between nearly equal variants less sensitive to a noisy round
    auto time_rounds = [&](const std::function<exa_status()> &call, int reps, float *best_ms) -> exa_status {
        if (exa_status e = call()) return e;
        float bm = 1e30f;
        for (int round = 0; round < 3; round++) {
            CR(cudaEventRecord(e0, m->stream));
            for (int r = 0; r < reps; r++)
                if (exa_status e = call()) return e;
            CR(cudaEventRecord(e1, m->stream));
            CR(cudaEventSynchronize(e1));
            float ms = 0;
            CR(cudaEventElapsedTime(&ms, e0, e1));
            bm = std::min(bm, ms);
        }
        *best_ms = bm;
        return EXA_OK;
    };
    double best = 1e30;
    int best_block = m->block, best_factor = 0;
    const int blocks[] = {64, 128, 256};
    auto variant = [&](int block, int minb, bool byp, int pf, bool lazy = false) {
        exa::CodegenOptions cg;
        cg.precision = m->precision;
        cg.block = block;
        cg.min_blocks = minb;
        cg.bounds_check = m->bounds_check;
        cg.by_pattern = byp;
        cg.prefetch = pf;
        cg.lazy_loads = lazy;
        cg.fused_step = m->fused_step;
        return cg;
    };
    {
        std::vector<exa::CodegenOptions> v;
        for (int B : blocks) v.push_back(variant(B, 0, m->by_pattern, m->prefetch, m->lazy_loads));
        precompile(m, v);
    }
    for (int B : blocks) {
        if (exa_status e = setup_kernels(m, B)) return e;
        CR(S.get(&part, std::max(m->ntiles[exa::M_ALL], 1)));
        ExaOut o{};
        o.obj_part = part;
        o.c = m->d_cbuf;
        o.abuf = m->d_abuf;
        o.gbuf = m->d_gbuf;
        o.jac = m->d_jbuf;
        o.hess = m->d_hbuf;
        for (int factor : {0, 1, 2, 4}) {
            if (exa_status e = apply_grid(m, factor)) return e;
            if (factor > 0 && m->grid[exa::M_ALL] == m->ntiles[exa::M_ALL]) continue;
            float ms = 0;
            if (exa_status e = time_rounds([&]() { return launch_eval(m, exa::M_ALL, x, y, 1.0, o); }, 5, &ms)) return e;
            if (ms < best) {
                best = ms;
                best_block = B;
                best_factor = factor;
            }
        }
    }
    // register budget and emission order, searched together: launch bounds asking for 20 to 32
    // resident warps per SM (the compiler may spill) or none, with each pattern's arithmetic next to
    // its outputs or all of a group's arithmetic up front; a variant is kept only when the fused
    // kernel gets faster (the uncapped per-pattern variant was timed above)
    int best_minb = 0;
    // emission orders: 0 each pattern's arithmetic next to its outputs, 1 up front, 2 as 0 with
    // each pattern's inputs loaded one pattern ahead
    const int init_order = m->by_pattern ? (m->lazy_loads ? 2 : 0) : 1;
    int best_order = init_order;
    {
        std::vector<exa::CodegenOptions> v;
        for (int order = 0; order < 3; order++)
            for (int warps : {0, 20, 24, 28, 32}) {
                const int minb = warps * 32 / best_block;
                if (minb <= 32 && (warps == 0 || minb >= 1))
                    v.push_back(variant(best_block, minb, order != 1, m->prefetch, order == 2));
            }
        precompile(m, v);
    }
    for (int order = 0; order < 3; order++) {
        const bool byp = order != 1;
        int last_minb = -1;
        for (int warps : {0, 20, 24, 28, 32}) {
            const int minb = warps * 32 / best_block;
            if (minb > 32 || minb == last_minb || (warps && minb < 1)) continue;
            last_minb = minb;
            if (order == init_order && minb == 0) continue;  // the variant timed by the search above
            m->by_pattern = byp;
            m->lazy_loads = order == 2;
            if (exa_status e = setup_kernels(m, best_block, minb)) return e;
            if (minb && m->regs[exa::M_ALL] * best_block * minb > 65536 + 1) continue;  // bound not honoured
            int occ = 0;
            CR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)m->fn[exa::M_ALL], best_block,
                                                             (size_t)m->dsmem[exa::M_ALL]));
            if (occ < minb) continue;
            CR(S.get(&part, std::max(m->ntiles[exa::M_ALL], 1)));
            ExaOut o{};
            o.obj_part = part;
            o.c = m->d_cbuf;
            o.abuf = m->d_abuf;
            o.gbuf = m->d_gbuf;
            o.jac = m->d_jbuf;
            o.hess = m->d_hbuf;
            if (exa_status e = apply_grid(m, best_factor)) return e;
            float ms = 0;
            if (exa_status e = time_rounds([&]() { return launch_eval(m, exa::M_ALL, x, y, 1.0, o); }, 5, &ms)) return e;
            if (ms < best) {
                best = ms;
                best_minb = minb;
                best_order = order;
            }
        }
    }
    m->by_pattern = best_order != 1;
    m->lazy_loads = best_order == 2;
    // L2 prefetch depth (staging of later tiles' inputs): none, data columns, or data columns and
    // the next tile's x and y lines; kept when the fused kernel gets faster
    const int init_pf = m->prefetch;
    int best_pf = init_pf;
    {
        std::vector<exa::CodegenOptions> v;
        for (int pf : {0, 1, 2})
            if (pf != init_pf) v.push_back(variant(best_block, best_minb, best_order != 1, pf, best_order == 2));
        precompile(m, v);
    }
    for (int pf : {0, 1, 2}) {
        if (pf == init_pf) continue;
        m->prefetch = pf;
        if (exa_status e = setup_kernels(m, best_block, best_minb)) return e;
        if (exa_status e = apply_grid(m, best_factor)) return e;
        CR(S.get(&part, std::max(m->ntiles[exa::M_ALL], 1)));
        ExaOut o{};
        o.obj_part = part;
        o.c = m->d_cbuf;
        o.abuf = m->d_abuf;
        o.gbuf = m->d_gbuf;
        o.jac = m->d_jbuf;
        o.hess = m->d_hbuf;
        float ms = 0;
        if (exa_status e = time_rounds([&]() { return launch_eval(m, exa::M_ALL, x, y, 1.0, o); }, 5, &ms)) return e;
        if (ms < best) {
            best = ms;
            best_pf = pf;
        }
    }
    m->prefetch = best_pf;
    // two warp sets per instance (fewer values live per thread, so a register cap allows more
    // warps): a fresh search over the register cap, kept when the fused kernel gets faster
    const int init_lanes = m->lanes;
    int best_lanes = init_lanes, best_lminb = best_minb;
    if (init_lanes == 1 && best_block % 64 == 0) {
        std::vector<exa::CodegenOptions> v;
        const std::vector<int> warps_l = {0, 24, 32, 40, 48};
        for (int warps : warps_l) {
            const int minb = warps * 32 / best_block;
            if (minb <= 32 && (warps == 0 || minb >= 1)) {
                exa::CodegenOptions cg = variant(best_block, minb, best_order != 1, 0, best_order == 2);
                cg.lanes = 2;
                v.push_back(cg);
            }
        }
        precompile(m, v);
        m->lanes = 2;
        const int keep_pf = m->prefetch;
        m->prefetch = 0;
        int last_minb = -1;
        for (int warps : warps_l) {
            const int minb = warps * 32 / best_block;
            if (minb > 32 || minb == last_minb || (warps && minb < 1)) continue;
            last_minb = minb;
            if (exa_status e = setup_kernels(m, best_block, minb)) return e;
            if (minb && m->regs[exa::M_ALL] * best_block * minb > 65536 + 1) continue;
            if (exa_status e = apply_grid(m, best_factor)) return e;
            CR(S.get(&part, std::max(m->ntiles[exa::M_ALL], 1)));
            ExaOut o{};
            o.obj_part = part;
            o.c = m->d_cbuf;
            o.abuf = m->d_abuf;
            o.gbuf = m->d_gbuf;
            o.jac = m->d_jbuf;
            o.hess = m->d_hbuf;
            float ms = 0;
            if (exa_status e = time_rounds([&]() { return launch_eval(m, exa::M_ALL, x, y, 1.0, o); }, 5, &ms)) return e;
            if (ms < best) {
                best = ms;
                best_lanes = 2;
                best_lminb = minb;
            }
        }
        m->prefetch = best_lanes == 2 ? 0 : keep_pf;
    }
    m->lanes = best_lanes;
    if (best_lanes == 2) best_minb = best_lminb;
    // staging depth 1 (the next tile's inputs copied into shared memory while the current tile
    // computes): the two buffers bound occupancy below what a register cap would, so the variant
    // has no cap; the persistent grid (which the staging needs: a CTA with one tile has nothing to
    // overlap) is searched afresh; kept when the fused kernel gets faster
    const int init_stage = m->stage;
    int best_stage = init_stage, best_sminb = best_minb, best_sfactor = best_factor;
    if (init_stage == 0 && m->lanes == 1 && !m->bounds_check) {
        const std::vector<int> warps_s = {0};
        std::vector<exa::CodegenOptions> v;
        for (int warps : warps_s) {
            const int minb = warps * 32 / best_block;
            if (minb <= 32 && (warps == 0 || minb >= 1)) {
                exa::CodegenOptions cg = variant(best_block, minb, best_order != 1, 0, best_order == 2);
                cg.stage = 1;
                v.push_back(cg);
            }
        }
        precompile(m, v);
        m->stage = 1;
        const int keep_pf = m->prefetch;
        m->prefetch = 0;
        int last_minb = -1;
        for (int warps : warps_s) {
            const int minb = warps * 32 / best_block;
            if (minb > 32 || minb == last_minb || (warps && minb < 1)) continue;
            last_minb = minb;
            if (exa_status e = setup_kernels(m, best_block, minb)) return e;
            if (minb && m->regs[exa::M_ALL] * best_block * minb > 65536 + 1) continue;
            CR(S.get(&part, std::max(m->ntiles[exa::M_ALL], 1)));
            ExaOut o{};
            o.obj_part = part;
            o.c = m->d_cbuf;
            o.abuf = m->d_abuf;
            o.gbuf = m->d_gbuf;
            o.jac = m->d_jbuf;
            o.hess = m->d_hbuf;
            for (int factor : {1, 2, 4}) {
                if (exa_status e = apply_grid(m, factor)) return e;
                if (m->grid[exa::M_ALL] == m->ntiles[exa::M_ALL] && factor > 1) continue;
                float ms = 0;
                if (exa_status e = time_rounds([&]() { return launch_eval(m, exa::M_ALL, x, y, 1.0, o); }, 5, &ms)) return e;
                if (ms < best) {
                    best = ms;
                    best_stage = 1;
                    best_sminb = minb;
                    best_sfactor = factor;
                }
            }
        }
        m->prefetch = best_stage ? 0 : keep_pf;
    }
    m->stage = best_stage;
    if (best_stage && !init_stage) {
        best_minb = best_sminb;
        best_factor = best_sfactor;
    }
    if (exa_status e = setup_kernels(m, best_block, best_minb)) return e;
    if (exa_status e = apply_grid(m, best_factor)) return e;
    m->tune_ms = best / 5.0;
    // exa_eval_all with every output: one kernel or first/second order split, CSC by a separate
    // permutation kernel or scattered by the evaluation kernel
    double *f = nullptr, *g = nullptr, *jc = nullptr, *hc = nullptr;
    CR(S.get(&f, 1));
    CR(S.get(&g, m->nvar));
    CR(S.get(&jc, m->nnzj_csc));
    CR(S.get(&hc, m->nnzh_csc));
    double best_step = 1e30;
    bool best_split = false, best_direct = false, best_hc = m->use_hcomp;
    int best_chunks = m->nchunks, best_wave = m->wave_pct;
    const int init_wave = m->wave_pct;
    for (int nch : {1, 2, 4, 8, 16})
    for (int wave : {0, 75, 50})
    for (int hcv = 0; hcv < (m->has_hcomp ? 2 : 1); hcv++)
    for (int split = 0; split < 2; split++)
        for (int direct = 0; direct < 2; direct++) {
            if (direct && m->nnzj_csc != m->nnzj && m->nnzh_csc != m->nnzh) continue;
            if (nch > m->nb || (m->chunks_fixed && nch != best_chunks)) continue;
            // a partial-wave grid only pays when chunks give the reductions something to overlap
            if (m->wave_fixed ? wave != 0 : (wave && nch == 1)) continue;
            m->wave_pct = m->wave_fixed ? init_wave : wave;
            if (exa_status e = apply_grid(m, best_factor)) return e;
            set_chunks(m, nch);
            m->split_all = split;
            m->csc_direct = direct;
            m->use_hcomp = hcv;
            float ms = 0;
            if (exa_status e = time_rounds([&]() { return eval_all_launches(m, x, y, 1.0, f, g, m->d_cbuf, m->d_jbuf, m->d_hbuf, jc, hc); },
                                           3, &ms))
                return e;
            if (ms < best_step) {
                best_step = ms;
                best_split = split;
                best_direct = direct;
                best_hc = hcv;
                best_chunks = nch;
                best_wave = m->wave_pct;
            }
        }
    m->wave_pct = best_wave;
    if (exa_status e = apply_grid(m, best_factor)) return e;
    set_chunks(m, best_chunks);
    m->split_all = best_split;
    m->csc_direct = best_direct;
    m->use_hcomp = best_hc;
    // the register cap was chosen for the fused kernel; when the step runs first and second order
    // as two kernels, the cap is searched again with whole steps (the variants are compiled)
    if (best_split && m->lanes == 1) {
        int split_minb = m->min_blocks;
        for (int warps : {0, 20, 24, 28, 32}) {
            const int minb = warps * 32 / best_block;
            if (minb > 32 || (warps && minb < 1) || minb == m->min_blocks) continue;
            const int keep = m->min_blocks;
            if (exa_status e = setup_kernels(m, best_block, minb)) return e;
            int occ = 0;
            CR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)m->fn[exa::M_FIRST], best_block,
                                                             (size_t)m->dsmem[exa::M_FIRST]));
            if (minb && occ < minb) {
                if (exa_status e = setup_kernels(m, best_block, keep)) return e;
                if (exa_status e = apply_grid(m, best_factor)) return e;
                continue;
            }
            if (exa_status e = apply_grid(m, best_factor)) return e;
            float ms = 0;
            if (exa_status e = time_rounds([&]() { return eval_all_launches(m, x, y, 1.0, f, g, m->d_cbuf, m->d_jbuf, m->d_hbuf, jc, hc); },
                                           3, &ms))
                return e;
            if (ms < best_step) {
                best_step = ms;
                split_minb = minb;
            }
            if (exa_status e = setup_kernels(m, best_block, keep)) return e;
            if (exa_status e = apply_grid(m, best_factor)) return e;
        }
        if (split_minb != m->min_blocks) {
            if (exa_status e = setup_kernels(m, best_block, split_minb)) return e;
            if (exa_status e = apply_grid(m, best_factor)) return e;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return EXA_OK;
}

// Fused groups: patterns whose instance counts are equal in every member are evaluated by one
// thread per instance (declaration order), so loads and subexpressions they share are computed
// once.  Data columns that are the same host array in every member become one group column;
// constants that differ between members get one descriptor slot per distinct value vector.  A
// group is closed when it would exceed 16 patterns, columns or constant slots.
exa_status build_groups(exa_model *m, const exa_model_desc *const *descs, int nb, bool fuse) {
    const int np = (int)m->pats.size();
    struct Acc {
        std::vector<long long> ninst;
        std::map<std::pair<int, std::vector<const void *>>, int> cols;
        std::map<std::vector<long long>, int> ics;
        std::map<std::vector<uint64_t>, int> fcs;
    };
    std::vector<Acc> acc;
    m->groups.clear();
    for (int p = 0; p < np; p++) {
        exa::Pattern &P = m->pats[p];
        std::vector<long long> ninst;
        for (int b = 0; b < nb; b++) ninst.push_back(descs[b]->patterns[p].n_inst);
        // keys of this pattern's columns and member-varying constants
        std::vector<std::pair<int, std::vector<const void *>>> colkeys;
        for (int f = 0; f < (int)P.ftype.size(); f++) {
            std::vector<const void *> ptrs;
            for (int b = 0; b < nb; b++) ptrs.push_back(descs[b]->patterns[p].fields[f].data);
            colkeys.push_back({P.ftype[f], ptrs});
        }
        std::vector<std::pair<int, std::vector<long long>>> ikeys;
        for (int i = 0; i < (int)P.ix.size(); i++) {
            if (P.ix[i].op != EXA_I_CONST) continue;
            std::vector<long long> vals;
            bool differ = false;
            for (int b = 0; b < nb; b++) {
                vals.push_back(descs[b]->patterns[p].inodes[i].ival);
                differ = differ || vals.back() != vals[0];
            }
            if (differ) ikeys.push_back({i, vals});
        }
        std::vector<std::pair<int, std::vector<uint64_t>>> fkeys;
        for (int i = 0; i < (int)P.v.size(); i++) {
            if (P.v[i].op != EXA_V_CONST) continue;
            std::vector<uint64_t> vals;
            bool differ = false;
            for (int b = 0; b < nb; b++) {
                uint64_t u;
                std::memcpy(&u, &descs[b]->patterns[p].vnodes[i].fval, 8);
                vals.push_back(u);
                differ = differ || vals.back() != vals[0];
            }
            if (differ) fkeys.push_back({i, vals});
        }
        if (colkeys.size() > EXA_MAXF || ikeys.size() > 16 || fkeys.size() > 16)
            return fail(m, EXA_E_UNSUPPORTED, "pattern " + std::to_string(p) +
                                                  ": more than 16 data columns or member-varying constants");
        int gi = -1;
        if (fuse) {
            for (int g = (int)acc.size() - 1; g >= 0 && gi < 0; g--) {
                if (acc[g].ninst != ninst || m->groups[g].pats.size() >= EXA_MAXG) continue;
                std::set<std::pair<int, std::vector<const void *>>> c;
                for (auto &kv : acc[g].cols) c.insert(kv.first);
                for (auto &k : colkeys) c.insert(k);
                std::set<std::vector<long long>> ic;
                for (auto &kv : acc[g].ics) ic.insert(kv.first);
                for (auto &k : ikeys) ic.insert(k.second);
                std::set<std::vector<uint64_t>> fc;
                for (auto &kv : acc[g].fcs) fc.insert(kv.first);
                for (auto &k : fkeys) fc.insert(k.second);
                if (c.size() <= EXA_MAXF && ic.size() <= 16 && fc.size() <= 16) gi = g;
                break;  // only the most recent group with these instance counts is extended
            }
        }
        if (gi < 0) {
            gi = (int)acc.size();
            acc.push_back(Acc{ninst, {}, {}, {}});
            m->groups.emplace_back();
        }
        exa::Group &G = m->groups[gi];
        Acc &A = acc[gi];
        G.pats.push_back(p);
        std::vector<int> fmap;
        for (auto &k : colkeys) {
            auto r = A.cols.emplace(k, (int)A.cols.size());
            if (r.second) G.ftype.push_back(k.first);
            fmap.push_back(r.first->second);
        }
        G.field.push_back(fmap);
        P.ivary.clear();
        P.fvary.clear();
        for (auto &k : ikeys) P.ivary[k.first] = A.ics.emplace(k.second, (int)A.ics.size()).first->second;
        for (auto &k : fkeys) P.fvary[k.first] = A.fcs.emplace(k.second, (int)A.fcs.size()).first->second;
        G.nic = (int)A.ics.size();
        G.nfc = (int)A.fcs.size();
    }
    for (auto &G : m->groups) exa::finalize_group(G, m->pats);
    return EXA_OK;
}

exa_status create_impl(const exa_model_desc *const *descs, int nb, const exa_options *opt, exa_model *m) {
    auto t0 = std::chrono::steady_clock::now();
    exa_options o{};
    if (opt) o = *opt;
    if (o.precision != EXA_FP64 && o.precision != EXA_MIXED_FP32) return fail(m, EXA_E_INVALID, "unknown precision");
    
    m->precision = o.precision;
    m->device = o.device;
    m->bounds_check = (o.flags & EXA_FLAG_BOUNDS_CHECK) != 0;
    m->use_graphs = (o.flags & EXA_FLAG_NO_GRAPH) == 0;
    m->block = o.block_threads ? o.block_threads : 128;
    if (m->block % 32 || m->block < 32 || m->block > 1024) return fail(m, EXA_E_INVALID, "block_threads must be a multiple of 32 in [32, 1024]");
    if ((o.flags & EXA_FLAG_LANES2) && m->block % 64)
        return fail(m, EXA_E_INVALID, "EXA_FLAG_LANES2 needs block_threads a multiple of 64");
    if (o.grid_factor < -1 || o.grid_factor > 64) return fail(m, EXA_E_INVALID, "grid_factor must be in [-1, 64]");
    if (o.min_blocks < 0 || o.min_blocks > 32) return fail(m, EXA_E_INVALID, "min_blocks must be in [0, 32]");
    if (o.chunks < 0 || o.chunks > 16) return fail(m, EXA_E_INVALID, "chunks must be in [0, 16]");
    if (o.wave_pct < 0 || o.wave_pct > 99) return fail(m, EXA_E_INVALID, "wave_pct must be in [0, 99]");
    m->wave_pct = o.wave_pct;
    m->wave_fixed = o.wave_pct != 0;
    m->split_all = (o.flags & EXA_FLAG_SPLIT) != 0;
    m->by_pattern = (o.flags & EXA_FLAG_UPFRONT) == 0;
    m->csc_direct = (o.flags & EXA_FLAG_CSC_SCATTER) != 0;
    m->prefetch = (o.flags & EXA_FLAG_PF_GATHERS) ? 2 : (o.flags & EXA_FLAG_PF_COLUMNS) ? 1 : 0;
    m->lanes = (o.flags & EXA_FLAG_LANES2) ? 2 : 1;
    m->lazy_loads = (o.flags & EXA_FLAG_LAZY_LOADS) != 0;
    m->stage = (o.flags & EXA_FLAG_STAGE_SMEM) != 0 && !m->bounds_check;
    m->host_serial = (o.flags & EXA_FLAG_HOST_SERIAL) != 0;
    m->fused_step = (o.flags & EXA_FLAG_FUSED_STEP) != 0;
    if (m->fused_step && (m->stage || m->lanes > 1 || m->prefetch))
        return fail(m, EXA_E_INVALID, "EXA_FLAG_FUSED_STEP excludes staging, EXA_FLAG_LANES2 and the prefetch flags");
    if (m->fused_step && m->precision != EXA_FP64)
        return fail(m, EXA_E_INVALID, "EXA_FLAG_FUSED_STEP is for FP64 models");
    if (m->lazy_loads && !m->by_pattern) return fail(m, EXA_E_INVALID, "EXA_FLAG_LAZY_LOADS excludes EXA_FLAG_UPFRONT");
    if (m->lanes > 1 && m->prefetch) return fail(m, EXA_E_INVALID, "EXA_FLAG_LANES2 excludes the prefetch flags");
    if ((o.flags & EXA_FLAG_STAGE_SMEM) && (m->lanes > 1 || m->prefetch))
        return fail(m, EXA_E_INVALID, "EXA_FLAG_STAGE_SMEM excludes EXA_FLAG_LANES2 and the prefetch flags");
    if (nb < 1) return fail(m, EXA_E_INVALID, "empty batch");
    for (int b = 0; b < nb; b++) {
        const exa_model_desc *d = descs[b];
        if (!d) return fail(m, EXA_E_INVALID, "NULL model descriptor");
        if (d->nvar < 0 || d->ncon < 0 || d->npar < 0 || d->n_patterns < 0) return fail(m, EXA_E_INVALID, "negative size");
        if (d->n_patterns > 0 && !d->patterns) return fail(m, EXA_E_INVALID, "NULL pattern array");
        if (d->npar > 0 && !d->theta) return fail(m, EXA_E_INVALID, "NULL theta");
        if (d->n_patterns != descs[0]->n_patterns) return fail(m, EXA_E_INVALID, "batch members differ in pattern count");
        for (int p = 0; p < d->n_patterns; p++) {
            const exa_pattern_desc &pd = d->patterns[p];
            if ((pd.n_vnodes > 0 && !pd.vnodes) || (pd.n_inodes > 0 && !pd.inodes) || (pd.n_fields > 0 && !pd.fields))
                return fail(m, EXA_E_INVALID, "NULL node or field array");
            if (pd.n_vnodes < 0 || pd.n_inodes < 0 || pd.n_fields < 0) return fail(m, EXA_E_INVALID, "negative node count");
            for (int f = 0; f < pd.n_fields; f++)
                if (pd.n_inst > 0 && !pd.fields[f].data) return fail(m, EXA_E_INVALID, "NULL data column");
            if (b > 0 && !same_shape(pd, descs[0]->patterns[p]))
                return fail(m, EXA_E_INVALID, "batch members must share the same pattern trees");
        }
    }
    CR(cudaSetDevice(m->device));
    int major = 0, minor = 0;
    CR(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, m->device));
    CR(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, m->device));
    if (major != 10 || minor != 3)
        return fail(m, EXA_E_UNSUPPORTED, "this build targets sm_103a (GB300); device is sm_" +
                                                 std::to_string(major) + std::to_string(minor));

    // patterns from member 0 (the IR is shared)
    const exa_model_desc &d0 = *descs[0];
    const int np = d0.n_patterns;
    if (exa_status e = load_patterns(d0, m)) return e;
    // every member must identify variable references the same way as member 0
    for (int p = 0; p < np && nb > 1; p++) {
        const exa::Pattern &P = m->pats[p];
        const std::vector<int> ref = exa::symbol_partition(P, P.ix);
        for (int b = 1; b < nb; b++) {
            const exa_pattern_desc &pd = descs[b]->patterns[p];
            std::vector<exa::INode> ix;
            for (int i = 0; i < pd.n_inodes; i++)
                ix.push_back({pd.inodes[i].op, pd.inodes[i].a, pd.inodes[i].b, pd.inodes[i].ival});
            if (exa::symbol_partition(P, ix) != ref)
                return fail(m, EXA_E_INVALID, "batch members of pattern " + std::to_string(p) +
                                                  " identify variable references differently");
        }
    }
    if (exa_status e = build_groups(m, descs, nb, (o.flags & EXA_FLAG_NO_FUSE) == 0)) return e;
    const int ng = (int)m->groups.size();

    // per-member sizes and offsets; validate row blocks
    m->nb = nb;
    m->xoff.assign(nb + 1, 0); m->coff.assign(nb + 1, 0); m->joff.assign(nb + 1, 0); m->hoff.assign(nb + 1, 0);
    std::vector<i64> goff(nb + 1, 0), aoff(nb + 1, 0), poff(nb + 1, 0);
    struct PatOff { i64 n_inst, rbase, rlimit, jbase, hbase, gbase, abase; };
    std::vector<PatOff> po((size_t)nb * np);
    for (int b = 0; b < nb; b++) {
        const exa_model_desc &d = *descs[b];
        if (d.nvar >= (1LL << 31) || d.ncon >= (1LL << 31)) return fail(m, EXA_E_INVALID, "size too large");
        std::vector<int> covered(d.ncon, 0);
        i64 oj = 0, oh = 0, og = 0, oa = 0;
        for (int p = 0; p < np; p++) {
            const exa_pattern_desc &pd = d.patterns[p];
            const exa::Pattern &P = m->pats[p];
            if (pd.n_inst < 0 || pd.n_inst >= (1LL << 31)) return fail(m, EXA_E_INVALID, "bad instance count");
            if (P.kind == EXA_CON) {
                if (pd.row_base < 0 || pd.row_base + pd.n_inst > d.ncon) return fail(m, EXA_E_BOUNDS, "constraint block out of range");
                for (i64 r = pd.row_base; r < pd.row_base + pd.n_inst; r++)
                    if (covered[r]++) return fail(m, EXA_E_INVALID, "constraint blocks overlap");
            }
            if (P.kind == EXA_AUG) {
                if (pd.row_base < 0 || pd.row_limit < 0 || pd.row_base + pd.row_limit > d.ncon)
                    return fail(m, EXA_E_BOUNDS, "augmentation target block out of range");
                if (pd.n_inst > 0 && pd.row_limit == 0) return fail(m, EXA_E_INVALID, "augmentation target block is empty");
            }
            PatOff &pm = po[(size_t)b * np + p];
            pm = PatOff{pd.n_inst, pd.row_base, pd.row_limit, 0, 0, 0, 0};  // member offsets added below
            pm.hbase = oh; oh += pd.n_inst * P.nh();
            if (P.kind == EXA_OBJ) { pm.gbase = og; og += pd.n_inst * P.nj(); }
            else { pm.jbase = oj; oj += pd.n_inst * P.nj(); }
            if (P.kind == EXA_AUG) { pm.abase = oa; oa += pd.n_inst; }
        }
        for (i64 r = 0; r < d.ncon; r++)
            if (!covered[r]) return fail(m, EXA_E_INVALID, "every constraint row must belong to exactly one base constraint pattern");
        m->xoff[b + 1] = m->xoff[b] + d.nvar;
        m->coff[b + 1] = m->coff[b] + d.ncon;
        m->joff[b + 1] = m->joff[b] + oj;
        m->hoff[b + 1] = m->hoff[b] + oh;
        goff[b + 1] = goff[b] + og;
        aoff[b + 1] = aoff[b] + oa;
        poff[b + 1] = poff[b] + d.npar;
    }
    m->nvar = m->xoff[nb]; m->ncon = m->coff[nb]; m->nnzj = m->joff[nb]; m->nnzh = m->hoff[nb];
    m->nnzg = goff[nb]; m->naug = aoff[nb]; m->npar = poff[nb];
    if (m->nvar >= (1LL << 31) || m->ncon >= (1LL << 31) || m->nnzj >= (1LL << 31) || m->nnzh >= (1LL << 31) ||
        m->nnzg >= (1LL << 31) || m->naug >= (1LL << 31))
        return fail(m, EXA_E_INVALID, "model exceeds 2^31-1 variables, rows or nonzeros");

    // upload theta and data columns (identical host columns are uploaded once)
    CR(dalloc(m, &m->d_theta, m->npar));
    CR(dalloc(m, &m->d_status, 1));
    CR(cudaMemset(m->d_status, 0, sizeof(int)));
    std::vector<ExaPM> pms((size_t)nb * ng);
    for (int b = 0; b < nb; b++) {
        const exa_model_desc &d = *descs[b];
        if (d.npar) CR(cudaMemcpy(m->d_theta + poff[b], d.theta, sizeof(double) * d.npar, cudaMemcpyHostToDevice));
        std::map<const void *, const void *> uploaded;
        std::map<const void *, float *> uploaded32;
        for (int gi = 0; gi < ng; gi++) {
            const exa::Group &G = m->groups[gi];
            ExaPM &pm = pms[(size_t)b * ng + gi];
            std::memset(&pm, 0, sizeof pm);
            pm.n_inst = po[(size_t)b * np + G.pats[0]].n_inst;
            pm.xoff = m->xoff[b];
            pm.nvar_m = d.nvar;
            pm.poff = poff[b];
            pm.npar_m = d.npar;
            pm.grp = gi;
            pm.member = b;
            pm.hcbase = m->nnzhc;
            m->nnzhc += pm.n_inst * (i64)G.hc.size();
            for (size_t pos = 0; pos < G.pats.size(); pos++) {
                const int p = G.pats[pos];
                const exa::Pattern &P = m->pats[p];
                const exa_pattern_desc &pd = d.patterns[p];
                const PatOff &q = po[(size_t)b * np + p];
                pm.rbase[pos] = q.rbase + m->coff[b];
                pm.rlimit[pos] = q.rlimit;
                pm.jbase[pos] = q.jbase + m->joff[b];
                pm.hbase[pos] = q.hbase + m->hoff[b];
                pm.gbase[pos] = q.gbase + goff[b];
                pm.abase[pos] = q.abase + aoff[b];
                for (auto &kv : P.ivary) pm.ic[kv.second] = pd.inodes[kv.first].ival;
                for (auto &kv : P.fvary) pm.fc[kv.second] = pd.vnodes[kv.first].fval;
                for (int f = 0; f < pd.n_fields; f++) {
                    const int c = G.field[pos][f];
                    if (pm.f[c]) continue;
                    const void *h = pd.fields[f].data;
                    auto it = uploaded.find(h);
                    if (it != uploaded.end() && pd.n_inst > 0) { pm.f[c] = it->second; continue; }
                    size_t es = pd.fields[f].type == EXA_FIELD_I32 ? 4 : 8;
                    void *dp = nullptr;
                    CR(dalloc(m, (char **)&dp, (i64)(pd.n_inst * es)));
                    if (pd.n_inst) CR(cudaMemcpy(dp, h, es * pd.n_inst, cudaMemcpyHostToDevice));
                    pm.f[c] = dp;
                    uploaded[h] = dp;
                }
                if (m->precision == EXA_MIXED_FP32)  // FP32 copies of f64 columns
                    for (int f = 0; f < pd.n_fields; f++) {
                        const int c = G.field[pos][f];
                        if (pd.fields[f].type != EXA_FIELD_F64 || pm.f32[c]) continue;
                        const void *h = pd.fields[f].data;
                        auto it = uploaded32.find(h);
                        if (it != uploaded32.end() && pd.n_inst > 0) { pm.f32[c] = it->second; continue; }
                        std::vector<float> tmp((size_t)pd.n_inst);
                        for (i64 i = 0; i < pd.n_inst; i++) tmp[i] = (float)((const double *)h)[i];
                        float *dp = nullptr;
                        CR(dalloc(m, &dp, pd.n_inst));
                        if (pd.n_inst) CR(cudaMemcpy(dp, tmp.data(), sizeof(float) * pd.n_inst, cudaMemcpyHostToDevice));
                        pm.f32[c] = dp;
                        uploaded32[h] = dp;
                    }
            }
        }
    }
    CR(dalloc(m, &m->d_pm, (i64)pms.size()));
    CR(cudaMemcpy(m->d_pm, pms.data(), sizeof(ExaPM) * pms.size(), cudaMemcpyHostToDevice));

    m->h_pms = pms;
    if (exa_status e = setup_kernels(m, m->block, o.min_blocks)) return e;

    // structure pass on the device
    CR(dalloc(m, &m->d_jrow, m->nnzj));
    CR(dalloc(m, &m->d_jcol, m->nnzj));
    CR(dalloc(m, &m->d_hrow, m->nnzh));
    CR(dalloc(m, &m->d_hcol, m->nnzh));
    CR(dalloc(m, &m->d_gvar, m->nnzg));
    CR(dalloc(m, &m->d_arow, m->naug));
    m->has_hcomp = m->nnzhc < m->nnzh;
    m->use_hcomp = m->has_hcomp && !(o.flags & EXA_FLAG_NO_HCOMP);
    if (m->has_hcomp) {
        CR(dalloc(m, &m->d_hcrow, m->nnzhc));
        CR(dalloc(m, &m->d_hccol, m->nnzhc));
    }
    if (m->ntiles[exa::M_STRUCT]) {
        ExaOut out{};
        out.status = m->d_status;
        ExaStructOut so{m->d_jrow, m->d_jcol, m->d_hrow, m->d_hcol, m->d_gvar, m->d_arow,
                        m->has_hcomp ? m->d_hcrow : nullptr, m->has_hcomp ? m->d_hccol : nullptr, m->d_status};
        const double *nul = nullptr;
        double sigma = 0;
        int nt = m->ntiles[exa::M_STRUCT];
        int pfd = 0;
        void *args[] = {&m->d_tiles[exa::M_STRUCT], &nt, &m->d_pm, &nul, &nul, &m->d_theta, &sigma, &out, &so, &pfd};
        CR(cudaLaunchKernel((const void *)m->fn[exa::M_STRUCT], dim3(m->ntiles[exa::M_STRUCT]), dim3(m->block),
                            args, 0, m->stream));
        CR(cudaStreamSynchronize(m->stream));
        int st = 0;
        CR(cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st) return fail(m, EXA_E_BOUNDS, "a resolved variable, parameter or row index is out of range");
    }
    if (exa_status e = build_structure(m)) return e;
    if (exa_status e = build_member_bounds(m)) return e;
    set_chunks(m, o.chunks ? o.chunks : 1);
    m->chunks_fixed = o.chunks != 0;

    // work buffers
    CR(dalloc(m, &m->d_jbuf, m->nnzj));
    CR(dalloc(m, &m->d_hbuf, m->nnzh));
    CR(dalloc(m, &m->d_gbuf, m->nnzg));
    CR(dalloc(m, &m->d_abuf, m->naug));
    CR(dalloc(m, &m->d_cbuf, m->ncon));
    {  // objective partials: one per CTA, at most one per tile; sized for 32-instance tiles
        i64 maxt = 1;
        for (const ExaPM &pm : m->h_pms) maxt += (pm.n_inst + 31) / 32;
        CR(dalloc(m, &m->d_objpart, maxt));
        m->objpart_n = maxt;
    }
    const bool tune = !(o.flags & EXA_FLAG_NO_TUNE) && !o.block_threads && o.grid_factor == 0;
    if (tune)
        if (exa_status e = autotune(m)) return e;
    if (!tune || o.grid_factor != 0)
        if (exa_status e = apply_grid(m, std::max(o.grid_factor, 0))) return e;
    if (exa_status e = prepare_step(m)) return e;
    CR(cudaDeviceSynchronize());
    m->create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return EXA_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

const char *exa_create_error(void) { return g_create_err.c_str(); }

const char *exa_last_error(const exa_model *m) { return m ? m->err.c_str() : "NULL model"; }

exa_status exa_create_batch(const exa_model_desc *const *descs, int32_t nb, const exa_options *opt, exa_model **out) {
    if (!out) return EXA_E_INVALID;
    *out = nullptr;
    if (!descs) {
        g_create_err = "NULL descriptor array";
        return EXA_E_INVALID;
    }
    exa_model *m = new (std::nothrow) exa_model();
    if (!m) {
        g_create_err = "host allocation failed";
        return EXA_E_OOM;
    }
    exa_status s;
    try {
        s = create_impl(descs, nb, opt, m);
    } catch (const std::exception &e) {
        s = fail(m, EXA_E_OOM, std::string("host exception: ") + e.what());
    }
    if (s != EXA_OK) {
        g_create_err = m->err;
        free_all(m);
        delete m;
        return s;
    }
    g_create_err.clear();
    *out = m;
    return EXA_OK;
}

exa_status exa_create(const exa_model_desc *desc, const exa_options *opt, exa_model **out) {
    const exa_model_desc *d[1] = {desc};
    return exa_create_batch(d, 1, opt, out);
}

void exa_destroy(exa_model *m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    free_all(m);
    delete m;
}

exa_status exa_dims(const exa_model *m, int64_t *nvar, int64_t *ncon, int64_t *nnzj, int64_t *nnzh,
                    int64_t *nnzj_csc, int64_t *nnzh_csc) {
    if (!m) return EXA_E_INVALID;
    if (nvar) *nvar = m->nvar;
    if (ncon) *ncon = m->ncon;
    if (nnzj) *nnzj = m->nnzj;
    if (nnzh) *nnzh = m->nnzh;
    if (nnzj_csc) *nnzj_csc = m->nnzj_csc;
    if (nnzh_csc) *nnzh_csc = m->nnzh_csc;
    return EXA_OK;
}

exa_status exa_batch_offsets(const exa_model *m, int32_t *nb, int64_t *xoff, int64_t *coff, int64_t *joff,
                             int64_t *hoff) {
    if (!m) return EXA_E_INVALID;
    if (nb) *nb = m->nb;
    for (int b = 0; b <= m->nb; b++) {
        if (xoff) xoff[b] = m->xoff[b];
        if (coff) coff[b] = m->coff[b];
        if (joff) joff[b] = m->joff[b];
        if (hoff) hoff[b] = m->hoff[b];
    }
    return EXA_OK;
}

exa_status exa_set_theta(exa_model *m, const double *theta, int64_t npar) {
    if (exa_status e = check_model(m)) return e;
    if (npar != m->npar) return fail(m, EXA_E_INVALID, "theta must have npar = " + std::to_string(m->npar) + " values");
    if (!npar) return EXA_OK;
    if (!theta) return fail(m, EXA_E_INVALID, "NULL theta");
    // ordered on the model's stream; synchronized so that the caller's array is free on return
    CR(cudaMemcpyAsync(m->d_theta, theta, sizeof(double) * npar, cudaMemcpyHostToDevice, m->stream));
    CR(cudaStreamSynchronize(m->stream));
    return EXA_OK;
}

exa_status exa_set_stream(exa_model *m, void *stream) {
    if (!m) return EXA_E_INVALID;
    m->stream = (cudaStream_t)stream;
    return EXA_OK;
}

#define CHECK_PTRS(...)                                                                            \
    do {                                                                                           \
        const void *ps_[] = {__VA_ARGS__};                                                         \
        for (const void *p_ : ps_)                                                                 \
            if (!p_) return fail(m, EXA_E_INVALID, "NULL array argument");                         \
    } while (0)

exa_status exa_obj(exa_model *m, const double *x, double *f) {
    if (exa_status e = check_model(m)) return e;
    CHECK_PTRS(x, f);
    ExaOut o{};
    o.obj_part = m->d_objpart;
    if (exa_status e = launch_eval(m, exa::M_OBJ, x, nullptr, 0.0, o)) return e;
    k_obj_final<<<1, 1024, 0, m->stream>>>(m->d_objpart, eval_grid(m, exa::M_OBJ, m->ntiles[exa::M_OBJ]), f);
    CR(cudaGetLastError());
    return EXA_OK;
}

// ---- objective without a scratch allocation -------------------------------------------------
// Callers that cannot allocate device memory themselves (their memory is owned by another
// allocator, or they run where cudaMalloc is not allowed) still need somewhere to put the
// per-CTA partial sums of the two-stage objective reduction.  exa_obj_noalloc uses this fixed
// array, which every GPU that loads the library holds until the process exits, instead of any
// allocated buffer.  Each launch overwrites the partials it reads, so nothing has to start at
// zero; calls that overlap on one GPU (any model, any stream) share the array and race.
#define EXA_NOALLOC_MAX_PARTIALS 65536
static __device__ __align__(256) double g_noalloc_partials[EXA_NOALLOC_MAX_PARTIALS];

namespace {
// The array's name is a host-side stand-in in host code, not a device address.  Its address on the
// model's device is asked for on every call, with that device current (check_model made it so): a
// runtime query that allocates nothing, and that stays right if the module is loaded again at
// another address (after cudaDeviceReset, for instance).
exa_status noalloc_partials(exa_model *m, double **out) {
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
        return fail(m, EXA_E_CUDA, std::string("cudaGetSymbolAddress of the static objective scratch: ") +
                                       cudaGetErrorString(e));
    *out = p;
    return EXA_OK;
}
}  // namespace

exa_status exa_obj_noalloc(exa_model *m, const double *x, double *f) {
    if (exa_status e = check_model(m)) return e;
    CHECK_PTRS(x, f);
    // one partial per CTA of the objective kernel: one CTA per objective tile (ceil(instances /
    // block) per batch member and fused group), or fewer in a persistent grid, so the limit depends
    // on the launch shape, not on instances alone
    const int nparts = eval_grid(m, exa::M_OBJ, m->ntiles[exa::M_OBJ]);
    if (nparts > EXA_NOALLOC_MAX_PARTIALS)
        return fail(m, EXA_E_UNSUPPORTED,
                    "exa_obj_noalloc: the objective needs " + std::to_string(nparts) +
                        " partial sums (one per CTA of its launch, tiles of up to " + std::to_string(m->block) +
                        " instances); the static scratch holds at most " +
                        std::to_string(EXA_NOALLOC_MAX_PARTIALS));
    double *part = nullptr;
    if (exa_status e = noalloc_partials(m, &part)) return e;
    ExaOut o{};
    o.obj_part = part;
    if (exa_status e = launch_eval(m, exa::M_OBJ, x, nullptr, 0.0, o)) return e;
    k_obj_final<<<1, 1024, 0, m->stream>>>(part, nparts, f);
    CR(cudaGetLastError());
    return EXA_OK;
}

// dst[s] = sum over segment s of src[perm[q]] (q ascending), s < n.
static exa_status seg_sum(exa_model *m, const int *ptr, const int *perm, const double *src, double *dst, i64 n,
                          cudaStream_t st) {
    if (n <= 0) return EXA_OK;
    k_seg_sum_warp<false><<<grid_of(n, 256 * EXA_SEG_G), 256, 0, st>>>(ptr, perm, src, dst, nullptr, (int)n);
    CR(cudaGetLastError());
    return EXA_OK;
}

static exa_status csc_sum(exa_model *m, const CscSum &cs, const double *src, double *dst, cudaStream_t st) {
    if (cs.n <= 0) return EXA_OK;
    k_permute<<<grid_of(cs.n, 256 * EXA_ILP), 256, 0, st>>>(cs.first, src, dst, (long long)cs.n);
    CR(cudaGetLastError());
    if (cs.n_multi) {
        k_seg_sum_warp<true><<<grid_of(cs.n_multi, 256 * EXA_SEG_G), 256, 0, st>>>(cs.mptr, cs.mperm, src, dst, cs.mseg,
                                                                                  cs.n_multi);
        CR(cudaGetLastError());
    }
    return EXA_OK;
}

// csc_sum over CSC positions [p0, p1), whose multi-entry segments are mseg[i0 .. i1).
static exa_status csc_sum_range(exa_model *m, const CscSum &cs, const double *src, double *dst, int p0, int p1,
                                int i0, int i1, cudaStream_t st) {
    if (p1 > p0) {
        k_permute<<<grid_of(p1 - p0, 256 * EXA_ILP), 256, 0, st>>>(cs.first + p0, src, dst + p0, (long long)(p1 - p0));
        CR(cudaGetLastError());
    }
    if (i1 > i0) {
        k_seg_sum_warp<true><<<grid_of(i1 - i0, 256 * EXA_SEG_G), 256, 0, st>>>(cs.mptr + i0, cs.mperm, src, dst,
                                                                               cs.mseg + i0, i1 - i0);
        CR(cudaGetLastError());
    }
    return EXA_OK;
}

// Dense gradient from the gradient slots.  Compact form (most variables without a slot): zero fill,
// then sums over the variables that have slots only.
static exa_status grad_sum(exa_model *m, double *g, cudaStream_t st) {
    if (!m->nvar) return EXA_OK;
    if (!m->grad_compact) return seg_sum(m, m->d_gptr, m->d_gperm, m->d_gbuf, g, m->nvar, st);
    CR(cudaMemsetAsync(g, 0, sizeof(double) * m->nvar, st));
    if (m->n_gseg) {
        k_seg_sum_warp<true><<<grid_of(m->n_gseg, 256 * EXA_SEG_G), 256, 0, st>>>(m->d_gsegptr, m->d_gperm, m->d_gbuf, g,
                                                                                 m->d_gsegvar, m->n_gseg);
        CR(cudaGetLastError());
    }
    return EXA_OK;
}

exa_status exa_grad(exa_model *m, const double *x, double *g) {
    if (exa_status e = check_model(m)) return e;
    CHECK_PTRS(x, g);
    ExaOut o{};
    o.gbuf = m->d_gbuf;
    if (exa_status e = launch_eval(m, exa::M_GRAD, x, nullptr, 0.0, o)) return e;
    if (m->nvar) {
        if (exa_status e = grad_sum(m, g, m->stream)) return e;
    }
    return EXA_OK;
}

static exa_status aug_rows(exa_model *m, double *c, cudaStream_t st) {
    if (m->n_aug_rows) {
        k_seg_sum_warp<true><<<grid_of(m->n_aug_rows, 256 * EXA_SEG_G), 256, 0, st>>>(
            m->d_aptr, m->d_aperm, m->d_abuf, c, m->d_arows, m->n_aug_rows);
        CR(cudaGetLastError());
    }
    return EXA_OK;
}

exa_status exa_cons(exa_model *m, const double *x, double *c) {
    if (exa_status e = check_model(m)) return e;
    if (m->ncon == 0) return EXA_OK;
    CHECK_PTRS(x, c);
    ExaOut o{};
    o.c = c;
    o.abuf = m->d_abuf;
    if (exa_status e = launch_eval(m, exa::M_CON, x, nullptr, 0.0, o)) return e;
    return aug_rows(m, c, m->stream);
}

exa_status exa_jac_structure(const exa_model *mc, int32_t *rows, int32_t *cols) {
    exa_model *m = const_cast<exa_model *>(mc);
    if (exa_status e = check_model(m)) return e;
    if (!m->nnzj) return EXA_OK;
    CHECK_PTRS(rows, cols);
    CR(cudaMemcpyAsync(rows, m->d_jrow, sizeof(int) * m->nnzj, cudaMemcpyDeviceToDevice, m->stream));
    CR(cudaMemcpyAsync(cols, m->d_jcol, sizeof(int) * m->nnzj, cudaMemcpyDeviceToDevice, m->stream));
    return EXA_OK;
}

exa_status exa_hess_structure(const exa_model *mc, int32_t *rows, int32_t *cols) {
    exa_model *m = const_cast<exa_model *>(mc);
    if (exa_status e = check_model(m)) return e;
    if (!m->nnzh) return EXA_OK;
    CHECK_PTRS(rows, cols);
    CR(cudaMemcpyAsync(rows, m->d_hrow, sizeof(int) * m->nnzh, cudaMemcpyDeviceToDevice, m->stream));
    CR(cudaMemcpyAsync(cols, m->d_hcol, sizeof(int) * m->nnzh, cudaMemcpyDeviceToDevice, m->stream));
    return EXA_OK;
}

exa_status exa_jac_coord(exa_model *m, const double *x, double *vals) {
    if (exa_status e = check_model(m)) return e;
    if (!m->nnzj) return EXA_OK;
    CHECK_PTRS(x, vals);
    ExaOut o{};
    o.jac = vals;
    return launch_eval(m, exa::M_JAC, x, nullptr, 0.0, o);
}

exa_status exa_hess_coord(exa_model *m, const double *x, const double *y, double sigma, double *vals) {
    if (exa_status e = check_model(m)) return e;
    if (!m->nnzh) return EXA_OK;
    CHECK_PTRS(x, vals);
    if (m->ncon && !y) return fail(m, EXA_E_INVALID, "NULL y");
    ExaOut o{};
    o.hess = vals;
    return launch_eval(m, exa::M_HESS, x, y, sigma, o);
}

static exa_status csc_structure(exa_model *m, i64 nnz, i64 nnz_csc, const int *dcolptr, const int *drowval,
                                const int *dmap, int32_t *colptr, int32_t *rowval, int32_t *coo2csc) {
    CHECK_PTRS(colptr);
    CR(cudaMemcpyAsync(colptr, dcolptr, sizeof(int) * (m->nvar + 1), cudaMemcpyDeviceToDevice, m->stream));
    if (nnz_csc) {
        CHECK_PTRS(rowval);
        CR(cudaMemcpyAsync(rowval, drowval, sizeof(int) * nnz_csc, cudaMemcpyDeviceToDevice, m->stream));
    }
    if (nnz && coo2csc) CR(cudaMemcpyAsync(coo2csc, dmap, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, m->stream));
    return EXA_OK;
}

exa_status exa_jac_csc_structure(const exa_model *mc, int32_t *colptr, int32_t *rowval, int32_t *coo2csc) {
    exa_model *m = const_cast<exa_model *>(mc);
    if (exa_status e = check_model(m)) return e;
    return csc_structure(m, m->nnzj, m->nnzj_csc, m->d_jcolptr, m->d_jrowval, m->d_jcoo2csc, colptr, rowval, coo2csc);
}

exa_status exa_hess_csc_structure(const exa_model *mc, int32_t *colptr, int32_t *rowval, int32_t *coo2csc) {
    exa_model *m = const_cast<exa_model *>(mc);
    if (exa_status e = check_model(m)) return e;
    return csc_structure(m, m->nnzh, m->nnzh_csc, m->d_hcolptr, m->d_hrowval, m->d_hcoo2csc, colptr, rowval, coo2csc);
}

static exa_status scatter_csc(exa_model *m, const CscSum &cs, const int *perm, const double *coo, double *csc,
                              i64 n, i64 nnz, cudaStream_t st) {
    if (!n) return EXA_OK;
    if (n != nnz) return csc_sum(m, cs, coo, csc, st);
    k_permute<<<grid_of(n, 256 * EXA_ILP), 256, 0, st>>>(perm, coo, csc, (long long)n);
    CR(cudaGetLastError());
    return EXA_OK;
}

exa_status exa_jac_csc(exa_model *m, const double *x, double *vals_csc) {
    if (exa_status e = check_model(m)) return e;
    if (!m->nnzj) return EXA_OK;
    CHECK_PTRS(x, vals_csc);
    ExaOut o{};
    o.jac = m->d_jbuf;
    if (m->nnzj_csc == m->nnzj) {  // permutation: written directly by the evaluation kernel
        o.jac = nullptr;
        o.jcsc = vals_csc;
        o.jmap = m->d_jcoo2csc;
        return launch_eval(m, exa::M_JAC, x, nullptr, 0.0, o);
    }
    if (exa_status e = launch_eval(m, exa::M_JAC, x, nullptr, 0.0, o)) return e;
    return scatter_csc(m, m->sum_j, m->d_jperm, m->d_jbuf, vals_csc, m->nnzj_csc, m->nnzj, m->stream);
}

exa_status exa_hess_csc(exa_model *m, const double *x, const double *y, double sigma, double *vals_csc) {
    if (exa_status e = check_model(m)) return e;
    if (!m->nnzh) return EXA_OK;
    CHECK_PTRS(x, vals_csc);
    if (m->ncon && !y) return fail(m, EXA_E_INVALID, "NULL y");
    ExaOut o{};
    o.hess = m->d_hbuf;
    if (m->nnzh_csc == m->nnzh) {
        o.hess = nullptr;
        o.hcsc = vals_csc;
        o.hmap = m->d_hcoo2csc;
        return launch_eval(m, exa::M_HESS, x, y, sigma, o);
    }
    if (m->use_hcomp) {
        o.hess = nullptr;
        o.hcomp = m->d_hcbuf;
        if (exa_status e = launch_eval(m, exa::M_HESS_C, x, y, sigma, o)) return e;
        return csc_sum(m, m->sum_hc, m->d_hcbuf, vals_csc, m->stream);
    }
    if (exa_status e = launch_eval(m, exa::M_HESS, x, y, sigma, o)) return e;
    return scatter_csc(m, m->sum_h, m->d_hperm, m->d_hbuf, vals_csc, m->nnzh_csc, m->nnzh, m->stream);
}

// The side streams of exa_eval_all run at the highest priority, so that the reductions' CTAs are
// scheduled as soon as an evaluation kernel's CTAs retire instead of queueing behind the next one.
static cudaError_t side_stream(cudaStream_t *s) {
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, hi);
}

// Records timing event ev (ev_k0 or ev_k1) on the model stream: plainly, or as an event-record node
// while this library captures its own graph; not inside a capture the caller is making.
static exa_status record_eval_event(exa_model *m, cudaEvent_t *ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CR(cudaStreamIsCapturing(m->stream, &cs));
    const bool own_capture = cs != cudaStreamCaptureStatusNone && m->stream == m->cap_stream;
    if (cs != cudaStreamCaptureStatusNone && !own_capture) return EXA_OK;
    if (!*ev) CR(cudaEventCreate(ev));
    if (own_capture) CR(cudaEventRecordWithFlags(*ev, m->stream, cudaEventRecordExternal));
    else CR(cudaEventRecord(*ev, m->stream));
    if (ev == &m->ev_k1) m->ev_k_valid = true;
    return EXA_OK;
}

// exa_eval_all over member chunks: for every chunk, its evaluation kernel(s) on the model stream,
// then, on side stream 0 once that chunk's kernel has finished, its Jacobian CSC, Hessian CSC,
// gradient and constraint reductions over the chunk's own ranges of every output (members own
// contiguous ranges of variables, rows, tiles and CSC positions).  The evaluation of the next chunk
// overlaps these reductions.  The objective sum follows the last evaluation; the host copies of
// f, g, c follow the last reduction.  Same kernels, same per-element arithmetic as one chunk.
static exa_status eval_all_chunked(exa_model *m, const double *x, const double *y, double sigma, double *f, double *g,
                                   double *c, double *jac_csc, double *hess_csc, ExaOut o,
                                   Mode mode, Mode hmode, bool split, bool jdirect, bool hdirect, bool hcomp) {
    if (!m->ev_fork) CR(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
    for (int s = 0; s < 3; s++) {
        if (!m->side[s]) CR(side_stream(&m->side[s]));
        if (!m->ev_join[s]) CR(cudaEventCreateWithFlags(&m->ev_join[s], cudaEventDisableTiming));
    }
    for (int k = 0; k < m->nchunks; k++)
        if (!m->ev_chunk[k]) CR(cudaEventCreateWithFlags(&m->ev_chunk[k], cudaEventDisableTiming));
    cudaStream_t ps = m->side[0];
    const bool jside = jac_csc && !jdirect && m->nnzj_csc;
    const bool hside = (hcomp || (hess_csc && !hdirect)) && m->nnzh_csc;
    ExaOut o1 = o, o2{};
    if (split) {
        o1.hess = nullptr;
        o1.hcsc = nullptr;
        o1.hcomp = nullptr;
        o2.hess = o.hess;
        o2.hcsc = o.hcsc;
        o2.hmap = o.hmap;
        o2.hcomp = o.hcomp;
    }
    const Mode m1 = split ? exa::M_FIRST : mode;
    int nparts = 0;  // objective partials so far: each chunk's launch writes one per CTA after them
    for (int k = 0; k < m->nchunks; k++) {
        const int b0 = m->chunk_b[k], b1 = m->chunk_b[k + 1];
        if (m->pre_chunk)
            if (exa_status e = m->pre_chunk(k)) return e;
        ExaOut oc = split ? o1 : o;
        oc.obj_part = m->d_objpart + nparts;
        if (k == 0)
            if (exa_status e = record_eval_event(m, &m->ev_k0)) return e;
        if (exa_status e = launch_eval(m, m1, x, y, sigma, oc, m->mb_tile[m1][b0], m->mb_tile[m1][b1]))
            return e;
        if (m->mb_tile[m1][b1] > m->mb_tile[m1][b0]) nparts += eval_grid(m, m1, m->mb_tile[m1][b1] - m->mb_tile[m1][b0]);
        if (split)
            if (exa_status e = launch_eval(m, hmode, x, y, sigma, o2, m->mb_tile[hmode][b0], m->mb_tile[hmode][b1]))
                return e;
        if (k == m->nchunks - 1)
            if (exa_status e = record_eval_event(m, &m->ev_k1)) return e;
        CR(cudaEventRecord(m->ev_chunk[k], m->stream));
        CR(cudaStreamWaitEvent(ps, m->ev_chunk[k], 0));
        if (jside) {
            const int p0 = m->mb_jcsc[b0], p1 = m->mb_jcsc[b1];
            if (m->nnzj_csc == m->nnzj) {
                if (p1 > p0) {
                    k_permute<<<grid_of(p1 - p0, 256 * EXA_ILP), 256, 0, ps>>>(m->d_jperm + p0, o.jac, jac_csc + p0,
                                                                            (long long)(p1 - p0));
                    CR(cudaGetLastError());
                }
            } else if (exa_status e = csc_sum_range(m, m->sum_j, o.jac, jac_csc, p0, p1, m->mb_jmulti[b0],
                                                    m->mb_jmulti[b1], ps)) {
                return e;
            }
        }
        if (hside) {
            const int p0 = m->mb_hcsc[b0], p1 = m->mb_hcsc[b1];
            if (hcomp) {
                if (exa_status e = csc_sum_range(m, m->sum_hc, m->d_hcbuf, hess_csc, p0, p1, m->mb_hcmulti[b0],
                                                 m->mb_hcmulti[b1], ps))
                    return e;
            } else if (m->nnzh_csc == m->nnzh) {
                if (p1 > p0) {
                    k_permute<<<grid_of(p1 - p0, 256 * EXA_ILP), 256, 0, ps>>>(m->d_hperm + p0, o.hess, hess_csc + p0,
                                                                            (long long)(p1 - p0));
                    CR(cudaGetLastError());
                }
            } else if (exa_status e = csc_sum_range(m, m->sum_h, o.hess, hess_csc, p0, p1, m->mb_hmulti[b0],
                                                    m->mb_hmulti[b1], ps)) {
                return e;
            }
        }
        if (g && m->nvar) {
            const i64 v0 = m->xoff[b0], v1 = m->xoff[b1];
            if (!m->grad_compact) {
                if (v1 > v0) {
                    k_seg_sum_warp<false><<<grid_of(v1 - v0, 256 * EXA_SEG_G), 256, 0, ps>>>(
                        m->d_gptr + v0, m->d_gperm, m->d_gbuf, g + v0, nullptr, (int)(v1 - v0));
                    CR(cudaGetLastError());
                }
            } else {
                if (v1 > v0) CR(cudaMemsetAsync(g + v0, 0, sizeof(double) * (v1 - v0), ps));
                const int s0 = m->mb_gseg[b0], s1 = m->mb_gseg[b1];
                if (s1 > s0) {
                    k_seg_sum_warp<true><<<grid_of(s1 - s0, 256 * EXA_SEG_G), 256, 0, ps>>>(
                        m->d_gsegptr + s0, m->d_gperm, m->d_gbuf, g, m->d_gsegvar + s0, s1 - s0);
                    CR(cudaGetLastError());
                }
            }
        }
        if (c) {
            const int a0 = m->mb_arow[b0], a1 = m->mb_arow[b1];
            if (a1 > a0) {
                k_seg_sum_warp<true><<<grid_of(a1 - a0, 256 * EXA_SEG_G), 256, 0, ps>>>(
                    m->d_aptr + a0, m->d_aperm, m->d_abuf, c, m->d_arows + a0, a1 - a0);
                CR(cudaGetLastError());
            }
        }
        if (m->post_chunk)
            if (exa_status e = m->post_chunk(k)) return e;
    }
    if (f) {
        k_obj_final<<<1, 1024, 0, m->stream>>>(m->d_objpart, nparts, f);
        CR(cudaGetLastError());
    }
    CR(cudaEventRecord(m->ev_join[0], ps));
    CR(cudaStreamWaitEvent(m->stream, m->ev_join[0], 0));
    return EXA_OK;
}

// Work queue of the fused step for kernel index i (0: exa_step over the M_ALL tiles, 1: exa_step_b
// over the M_ALL_B tiles): every evaluation tile in member order, and each member's reductions
// (Jacobian CSC, Hessian CSC, gradient, constraint augmentations, cut into pieces a CTA takes in
// one go) placed two resident grids' worth of items (at most a quarter of the tiles) after that
// member's last tile, so that by the time a CTA takes one the tiles it waits for are normally done.  Rebuilt when the tile lists or
// the launch shape change.
static exa_status build_step(exa_model *m, int i) {
    const Mode mode = i ? exa::M_ALL_B : exa::M_ALL;
    const int nb = m->nb;
    int sms = 0, occ = 0;
    CR(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    CR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)m->fn_step[i], m->block, 0));
    const std::vector<ExaTile> &tiles = m->h_tiles[mode];
    std::vector<int> need(nb, 0);
    for (int b = 0; b < nb; b++) need[b] = m->mb_tile[mode][b + 1] - m->mb_tile[mode][b];
    // reductions of member b: (kind, first, end) pieces
    auto pieces = [&](int b, std::vector<ExaTask> &out) {
        auto cut = [&](int kind, i64 lo, i64 hi, i64 step) {
            for (i64 p = lo; p < hi; p += step) out.push_back({kind, b, (int)p, (int)std::min(hi, p + step)});
        };
        cut(1, m->mb_jcsc[b], m->mb_jcsc[b + 1], m->nnzj_csc == m->nnzj ? 8192 : 2048);
        cut(2, m->mb_hcsc[b], m->mb_hcsc[b + 1], 2048);  // 2048 segments, or positions of a permutation
        if (m->grad_compact) cut(3, m->mb_gseg[b], m->mb_gseg[b + 1], 2048);
        else cut(3, m->xoff[b], m->xoff[b + 1], 2048);
        cut(4, m->mb_arow[b], m->mb_arow[b + 1], 2048);
    };
    std::vector<ExaTask> items;
    items.reserve(tiles.size() + 64 * (size_t)nb);
    const i64 grid_est = (i64)std::max(occ, 1) * sms;
    // items between a member's last tile and its reductions: two resident grids, or a quarter of
    // the tiles when there are few (so that small batches still interleave)
    const i64 lag = std::max<i64>(1, std::min<i64>(2 * grid_est, (i64)tiles.size() / 4));
    std::vector<std::pair<i64, int>> pending;  // (queue position from which due, member)
    int next_due = 0;
    for (int b = 0; b < nb; b++) {
        for (int t = m->mb_tile[mode][b]; t < m->mb_tile[mode][b + 1]; t++) {
            items.push_back({0, b, t, t + 1});
            while (next_due < (int)pending.size() && (i64)items.size() >= pending[next_due].first)
                pieces(pending[next_due++].second, items);
        }
        pending.push_back({(i64)items.size() + lag, b});
    }
    while (next_due < (int)pending.size()) pieces(pending[next_due++].second, items);
    if (items.size() > (size_t)INT32_MAX) return fail(m, EXA_E_UNSUPPORTED, "fused step queue too long");
    if (m->d_items[i]) cudaFree(m->d_items[i]);
    if (m->d_need[i]) cudaFree(m->d_need[i]);
    m->d_items[i] = nullptr;
    m->d_need[i] = nullptr;
    CR(cudaMalloc((void **)&m->d_items[i], sizeof(ExaTask) * std::max<size_t>(items.size(), 1)));
    CR(cudaMalloc((void **)&m->d_need[i], sizeof(int) * std::max(nb, 1)));
    if (!m->d_sctr) CR(cudaMalloc((void **)&m->d_sctr, sizeof(int) * (nb + 1)));
    if (!items.empty())
        CR(cudaMemcpy(m->d_items[i], items.data(), sizeof(ExaTask) * items.size(), cudaMemcpyHostToDevice));
    CR(cudaMemcpy(m->d_need[i], need.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
    m->nitems[i] = (int)items.size();
    // one CTA per resident slot (more would only queue), at most one objective partial per slot
    m->step_grid[i] = (int)std::max<i64>(1, std::min<i64>({grid_est, (i64)items.size(), m->objpart_n}));
    m->step_ready[i] = true;
    return EXA_OK;
}

// Builds the fused step's queues that are missing (outside any stream capture: they allocate).
static exa_status prepare_step(exa_model *m) {
    if (!m->fused_step) return EXA_OK;
    for (int i = 0; i < 2; i++)
        if (m->fn_step[i] && !m->step_ready[i])
            if (exa_status e = build_step(m, i)) return e;
    return EXA_OK;
}

// The fused step: one exa_step[_b] launch (tiles and reductions from one queue), then the objective.
static exa_status eval_fused_step(exa_model *m, int i, const double *x, const double *y, double sigma, ExaOut o,
                                  double *f, double *g, double *c, double *jac_csc, double *hess_csc, bool jdirect,
                                  bool hdirect, bool hcomp) {
    if (!m->step_ready[i])
        if (exa_status e = build_step(m, i)) return e;
    const Mode mode = i ? exa::M_ALL_B : exa::M_ALL;
    ExaStep st{};
    st.ctr = m->d_sctr;
    st.need = m->d_need[i];
    st.items = m->d_items[i];
    st.nitems = m->nitems[i];
    st.spin_limit = 1 << 22;  // polls of about 0.2 us or more: about a second at least
    for (ExaRed &r : st.r) r.how = -1;
    if (jac_csc && !jdirect && m->nnzj_csc) {
        st.r[0] = m->nnzj_csc == m->nnzj ? ExaRed{0, nullptr, m->d_jperm, nullptr, o.jac, jac_csc}
                                           : ExaRed{1, m->d_jsegptr, m->d_jperm, nullptr, o.jac, jac_csc};
    }
    if (hess_csc && !hdirect && m->nnzh_csc) {
        st.r[1] = hcomp                      ? ExaRed{1, m->d_hcsegptr, m->d_hcperm, nullptr, m->d_hcbuf, hess_csc}
                  : m->nnzh_csc == m->nnzh ? ExaRed{0, nullptr, m->d_hperm, nullptr, o.hess, hess_csc}
                                           : ExaRed{1, m->d_hsegptr, m->d_hperm, nullptr, o.hess, hess_csc};
    }
    if (g && m->nvar) {
        if (m->grad_compact) {
            CR(cudaMemsetAsync(g, 0, sizeof(double) * m->nvar, m->stream));
            st.r[2] = ExaRed{3, m->d_gsegptr, m->d_gperm, m->d_gsegvar, m->d_gbuf, g};
        } else {
            st.r[2] = ExaRed{2, m->d_gptr, m->d_gperm, nullptr, m->d_gbuf, g};
        }
    }
    if (c && m->n_aug_rows) st.r[3] = ExaRed{3, m->d_aptr, m->d_aperm, m->d_arows, m->d_abuf, c};
    CR(cudaMemsetAsync(m->d_sctr, 0, sizeof(int) * (m->nb + 1), m->stream));
    if (m->step_hold >= 0 && m->step_hold < m->nb) {
        // failure injection for one call: the member's count starts at -1, so it ends one short of
        // its tiles and its reductions' waits run out after a short bound
        CR(cudaMemsetAsync(m->d_sctr + 1 + m->step_hold, 0xff, sizeof(int), m->stream));
        st.spin_limit = 1 << 12;
        m->step_hold = -1;
    }
    o.status = m->d_status;
    ExaStructOut so{};
    so.status = m->d_status;
    const double *th = m->d_theta;
    const ExaTile *tiles = m->d_tiles[mode];
    int nt = m->ntiles[mode], pfd = 0;
    void *args[] = {&tiles, &nt, &m->d_pm, &x, &y, &th, &sigma, &o, &so, &pfd, &st};
    if (exa_status e = record_eval_event(m, &m->ev_k0)) return e;
    CR(cudaLaunchKernel((const void *)m->fn_step[i], dim3(m->step_grid[i]), dim3(m->block), args, 0, m->stream));
    if (exa_status e = record_eval_event(m, &m->ev_k1)) return e;
    if (f) {
        k_obj_final<<<1, 1024, 0, m->stream>>>(m->d_objpart, m->step_grid[i], f);
        CR(cudaGetLastError());
    }
    return EXA_OK;
}

static exa_status eval_all_launches(exa_model *m, const double *x, const double *y, double sigma, double *f,
                                    double *g, double *c, double *jac, double *hess, double *jac_csc,
                                    double *hess_csc) {
    const bool want_h = hess || hess_csc;
    ExaOut o{};
    o.obj_part = m->d_objpart;
    o.c = c ? c : m->d_cbuf;
    o.abuf = m->d_abuf;
    o.gbuf = m->d_gbuf;
    o.jac = jac ? jac : m->d_jbuf;
    o.hess = hess ? hess : m->d_hbuf;
    // a CSC without duplicates is a permutation of the COO slots: the evaluation kernel writes it
    // directly, and the COO copy is skipped when the caller did not ask for it
    const bool jdirect = m->csc_direct && jac_csc && m->nnzj_csc == m->nnzj;
    const bool hdirect = m->csc_direct && hess_csc && m->nnzh_csc == m->nnzh;
    if (jdirect) {
        o.jcsc = jac_csc;
        o.jmap = m->d_jcoo2csc;
        if (!jac) o.jac = nullptr;
    }
    if (hdirect) {
        o.hcsc = hess_csc;
        o.hmap = m->d_hcoo2csc;
        if (!hess) o.hess = nullptr;
    }
    const bool hcomp = hess_csc && !hdirect && m->use_hcomp;
    if (hcomp) {  // the CSC sums read the group-compressed entries instead of the COO slots
        o.hcomp = m->d_hcbuf;
        if (!hess) o.hess = nullptr;
    }
    // Hessian variant: COO slots, group-compressed sums for the CSC, or both
    const bool hcoo = o.hess != nullptr;
    Mode mode = !want_h ? exa::M_FIRST : (hcomp ? (hcoo ? exa::M_ALL_B : exa::M_ALL_C) : exa::M_ALL);
    const Mode hmode = hcomp ? (hcoo ? exa::M_HESS_B : exa::M_HESS_C) : exa::M_HESS;
    if (m->fused_step && m->nchunks == 1 && !(want_h && m->split_all) && want_h &&
        (mode == exa::M_ALL || mode == exa::M_ALL_B) && m->fn_step[mode == exa::M_ALL_B])
        return eval_fused_step(m, mode == exa::M_ALL_B, x, y, sigma, o, f, g, c, jac_csc, hess_csc, jdirect, hdirect,
                               hcomp);
    if (m->nchunks > 1)
        return eval_all_chunked(m, x, y, sigma, f, g, c, jac_csc, hess_csc, o, want_h ? mode : exa::M_FIRST,
                                hmode, want_h && m->split_all, jdirect, hdirect, hcomp);
    // Streams: the model stream runs the evaluation kernel(s); side 0 the Jacobian CSC, side 1 the
    // Hessian CSC, side 3 (split mode) the objective, gradient and constraint sums.  Each branch is
    // forked from and joined back into the model stream (parallel branches of the captured graph).
    // In split mode every first-order reduction starts as soon as the first-order kernel has run,
    // overlapping the second-order kernel: the reductions move bytes, the second-order kernel keeps
    // the FP64 pipe busy.
    const bool split = want_h && m->split_all;
    const bool jside = jac_csc && !jdirect && m->nnzj_csc, hside = (hcomp || (hess_csc && !hdirect)) && m->nnzh_csc;
    const bool forked = jside || hside || split;
    if (forked) {
        if (!m->ev_fork) CR(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
        if (!m->ev_first) CR(cudaEventCreateWithFlags(&m->ev_first, cudaEventDisableTiming));
        for (int s = 0; s < 4; s++) {
            if (!m->side[s]) CR(side_stream(&m->side[s]));
            if (!m->ev_join[s]) CR(cudaEventCreateWithFlags(&m->ev_join[s], cudaEventDisableTiming));
        }
    }
    if (split) {  // first order and second order as two kernels
        ExaOut o1 = o, o2{};
        o1.hess = nullptr;
        o1.hcsc = nullptr;
        o1.hcomp = nullptr;
        o2.hess = o.hess;
        o2.hcsc = o.hcsc;
        o2.hmap = o.hmap;
        o2.hcomp = o.hcomp;
        mode = exa::M_FIRST;
        if (exa_status e = record_eval_event(m, &m->ev_k0)) return e;
        if (exa_status e = launch_eval(m, exa::M_FIRST, x, y, sigma, o1)) return e;
        CR(cudaEventRecord(m->ev_first, m->stream));
        if (exa_status e = launch_eval(m, hmode, x, y, sigma, o2)) return e;
    } else {
        if (exa_status e = record_eval_event(m, &m->ev_k0)) return e;
        if (exa_status e = launch_eval(m, mode, x, y, sigma, o)) return e;
    }
    if (exa_status e = record_eval_event(m, &m->ev_k1)) return e;
    if (forked) CR(cudaEventRecord(m->ev_fork, m->stream));
    const cudaEvent_t first_done = split ? m->ev_first : m->ev_fork;  // first-order outputs final
    cudaStream_t rs = split ? m->side[3] : m->stream;                  // stream of the f, g, c sums
    if (split) CR(cudaStreamWaitEvent(rs, m->ev_first, 0));
    if (jside) {
        CR(cudaStreamWaitEvent(m->side[0], first_done, 0));
        if (exa_status e = scatter_csc(m, m->sum_j, m->d_jperm, o.jac, jac_csc, m->nnzj_csc, m->nnzj, m->side[0])) return e;
        CR(cudaEventRecord(m->ev_join[0], m->side[0]));
    }
    if (hside) {
        CR(cudaStreamWaitEvent(m->side[1], m->ev_fork, 0));
        if (hcomp) {
            if (exa_status e = csc_sum(m, m->sum_hc, m->d_hcbuf, hess_csc, m->side[1]))
                return e;
        } else if (exa_status e = scatter_csc(m, m->sum_h, m->d_hperm, o.hess, hess_csc, m->nnzh_csc, m->nnzh, m->side[1])) {
            return e;
        }
        CR(cudaEventRecord(m->ev_join[1], m->side[1]));
    }
    if (f) {
        k_obj_final<<<1, 1024, 0, rs>>>(m->d_objpart, eval_grid(m, mode, m->ntiles[mode]), f);
        CR(cudaGetLastError());
    }
    if (g && m->nvar)
        if (exa_status e = grad_sum(m, g, rs)) return e;
    if (c)
        if (exa_status e = aug_rows(m, c, rs)) return e;
    if (split) CR(cudaEventRecord(m->ev_join[3], m->side[3]));
    if (jside) CR(cudaStreamWaitEvent(m->stream, m->ev_join[0], 0));
    if (hside) CR(cudaStreamWaitEvent(m->stream, m->ev_join[1], 0));
    if (split) CR(cudaStreamWaitEvent(m->stream, m->ev_join[3], 0));
    return EXA_OK;
}

// exa_eval_all replays a CUDA graph of its launches (evaluation kernel plus the reductions it needs),
// captured once per argument tuple on a private stream and cached (at most 4 tuples, least recently
// used evicted).  When the model's stream is itself being captured, the launches go straight into
// the caller's capture instead.
static exa_status eval_all_cached(exa_model *m, const double *x, const double *y, double sigma, double *f, double *g,
                                  double *c, double *jac, double *hess, double *jac_csc, double *hess_csc) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CR(cudaStreamIsCapturing(m->stream, &cs));
    if (!m->use_graphs || cs != cudaStreamCaptureStatusNone || m->step_hold >= 0)
        return eval_all_launches(m, x, y, sigma, f, g, c, jac, hess, jac_csc, hess_csc);
    uint64_t sb;
    std::memcpy(&sb, &sigma, 8);
    const std::array<const void *, 10> key = {x, y, f, g, c, jac, hess, jac_csc, hess_csc, (const void *)(uintptr_t)sb};
    for (auto &ge : m->graphs)
        if (ge.key == key) {
            ge.last_use = ++m->graph_clock;
            CR(cudaGraphLaunch(ge.exec, m->stream));
            return EXA_OK;
        }
    if (!m->cap_stream) CR(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    if (exa_status e = prepare_step(m)) return e;  // allocations cannot happen inside the capture
    cudaStream_t user = m->stream;
    m->stream = m->cap_stream;
    CR(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
    exa_status st = eval_all_launches(m, x, y, sigma, f, g, c, jac, hess, jac_csc, hess_csc);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(m->cap_stream, &graph);
    m->stream = user;
    if (st != EXA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return fail(m, EXA_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    {  // kernels per replay of this graph (reported by exa_stat "graph_kernels")
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
            std::vector<cudaGraphNode_t> nodes(nn);
            int nk = 0;
            if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) nk++;
                }
            m->graph_kernels = nk;
        }
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(m, EXA_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    if (m->graphs.size() >= 4) {
        auto lru = std::min_element(m->graphs.begin(), m->graphs.end(),
                                    [](const exa_model::GraphEntry &a, const exa_model::GraphEntry &b) { return a.last_use < b.last_use; });
        cudaGraphExecDestroy(lru->exec);
        m->graphs.erase(lru);
    }
    m->graphs.push_back({key, exec, ++m->graph_clock});
    CR(cudaGraphLaunch(exec, m->stream));
    return EXA_OK;
}

exa_status exa_eval_all(exa_model *m, const double *x, const double *y, double sigma, double *f, double *g,
                        double *c, double *jac, double *hess, double *jac_csc, double *hess_csc) {
    if (exa_status e = check_model(m)) return e;
    CHECK_PTRS(x);
    if ((hess || hess_csc) && m->ncon && !y) return fail(m, EXA_E_INVALID, "NULL y");
    return eval_all_cached(m, x, y, sigma, f, g, c, jac, hess, jac_csc, hess_csc);
}

exa_status exa_eval_all_host(exa_model *m, const double *x, const double *y, double sigma, double *f, double *g,
                             double *c, double *jac, double *hess, double *jac_csc, double *hess_csc) {
    if (exa_status e = check_model(m)) return e;
    CHECK_PTRS(x);
    const bool want_h = hess || hess_csc;
    if (want_h && m->ncon && !y) return fail(m, EXA_E_INVALID, "NULL y");
    const i64 n[9] = {m->nvar, m->ncon, 1, m->nvar, m->ncon, m->nnzj, m->nnzh, m->nnzj_csc, m->nnzh_csc};
    double *arg[9] = {const_cast<double *>(x), const_cast<double *>(y), f, g, c, jac, hess, jac_csc, hess_csc};
    double *use[9] = {};
    bool staged[9] = {};
    bool any_out = false;
    for (int k = 0; k < 9; k++) {
        if (!arg[k]) continue;
        cudaPointerAttributes a{};
        CR(cudaPointerGetAttributes(&a, arg[k]));
        staged[k] = a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
        if (staged[k] && !m->d_host_io[k]) CR(dalloc(m, &m->d_host_io[k], n[k]));
        use[k] = staged[k] ? m->d_host_io[k] : arg[k];
        if (k >= 2) any_out = any_out || staged[k];
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CR(cudaStreamIsCapturing(m->stream, &cs));
    const int K = std::min(m->nb, 8);
    if (m->host_serial || K < 2 || !any_out || cs != cudaStreamCaptureStatusNone) {
        for (int k = 0; k < 2; k++)
            if (staged[k] && n[k] > 0)
                CR(cudaMemcpyAsync(use[k], arg[k], sizeof(double) * n[k], cudaMemcpyHostToDevice, m->stream));
        // the device-only graph, then every host output copied back on the model stream in turn
        if (exa_status e = eval_all_cached(m, use[0], use[1], sigma, use[2], use[3], use[4], use[5], use[6], use[7], use[8]))
            return e;
        for (int k = 2; k < 9; k++)
            if (staged[k] && n[k] > 0)
                CR(cudaMemcpyAsync(arg[k], use[k], sizeof(double) * n[k], cudaMemcpyDeviceToHost, m->stream));
        CR(cudaStreamSynchronize(m->stream));
        return EXA_OK;
    }
    // Batch pipeline over K member chunks (members are independent and their x, y, c, g, COO and CSC
    // entries are contiguous ranges): one stream copies every chunk's x and y in, the evaluation and
    // reductions of chunk k start when its inputs are there, and a second stream copies chunk k's
    // outputs back as soon as its reductions have run, so the link carries chunk k's outputs while
    // later chunks are still being copied in and evaluated.
    if (!m->h2d) CR(cudaStreamCreateWithFlags(&m->h2d, cudaStreamNonBlocking));
    if (!m->d2h) CR(cudaStreamCreateWithFlags(&m->d2h, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&m->ev_hstart, &m->ev_hdone})
        if (!*e) CR(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    for (int k = 0; k < K; k++)
        for (cudaEvent_t *e : {&m->ev_in[k], &m->ev_out[k]})
            if (!*e) CR(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    const int keep_chunks = m->nchunks;
    const std::vector<int> keep_b = m->chunk_b;
    set_chunks(m, K);
    const int nk = m->nchunks;
    // copies start after earlier work on the model stream
    CR(cudaEventRecord(m->ev_hstart, m->stream));
    CR(cudaStreamWaitEvent(m->h2d, m->ev_hstart, 0));
    CR(cudaStreamWaitEvent(m->d2h, m->ev_hstart, 0));
    // element ranges of chunk k: x and g over variables, y and c over rows, then the COO and CSC
    auto range = [&](int k, int which, i64 *lo, i64 *hi) {
        const int b0 = m->chunk_b[k], b1 = m->chunk_b[k + 1];
        switch (which) {
        case 0: case 3: *lo = m->xoff[b0]; *hi = m->xoff[b1]; break;
        case 1: case 4: *lo = m->coff[b0]; *hi = m->coff[b1]; break;
        case 5: *lo = m->joff[b0]; *hi = m->joff[b1]; break;
        case 6: *lo = m->hoff[b0]; *hi = m->hoff[b1]; break;
        case 7: *lo = m->mb_jcsc[b0]; *hi = m->mb_jcsc[b1]; break;
        case 8: *lo = m->mb_hcsc[b0]; *hi = m->mb_hcsc[b1]; break;
        default: *lo = *hi = 0; break;
        }
    };
    exa_status st = EXA_OK;
    for (int k = 0; k < nk && st == EXA_OK; k++) {
        for (int a = 0; a < 2; a++) {
            if (!staged[a]) continue;
            i64 lo, hi;
            range(k, a, &lo, &hi);
            if (hi > lo) {
                cudaError_t e = cudaMemcpyAsync(use[a] + lo, arg[a] + lo, sizeof(double) * (hi - lo), cudaMemcpyHostToDevice, m->h2d);
                if (e != cudaSuccess) st = fail(m, EXA_E_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
            }
        }
        if (st == EXA_OK) {
            cudaError_t e = cudaEventRecord(m->ev_in[k], m->h2d);
            if (e != cudaSuccess) st = fail(m, EXA_E_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
        }
    }
    m->pre_chunk = [&](int k) -> exa_status {
        CR(cudaStreamWaitEvent(m->stream, m->ev_in[k], 0));
        return EXA_OK;
    };
    m->post_chunk = [&](int k) -> exa_status {
        // chunk k's reductions ran on side stream 0 after its evaluation kernel
        CR(cudaEventRecord(m->ev_out[k], m->side[0]));
        CR(cudaStreamWaitEvent(m->d2h, m->ev_out[k], 0));
        for (int a = 3; a < 9; a++) {
            if (!staged[a]) continue;
            i64 lo, hi;
            range(k, a, &lo, &hi);
            if (hi > lo)
                CR(cudaMemcpyAsync(arg[a] + lo, use[a] + lo, sizeof(double) * (hi - lo), cudaMemcpyDeviceToHost, m->d2h));
        }
        return EXA_OK;
    };
    if (st == EXA_OK)
        st = eval_all_launches(m, use[0], use[1], sigma, use[2], use[3], use[4], use[5], use[6], use[7], use[8]);
    m->pre_chunk = nullptr;
    m->post_chunk = nullptr;
    m->nchunks = keep_chunks;
    m->chunk_b = keep_b;
    if (st != EXA_OK) {
        cudaStreamSynchronize(m->h2d);
        cudaStreamSynchronize(m->d2h);
        cudaStreamSynchronize(m->stream);
        return st;
    }
    // the objective after every chunk, then wait for the last copies
    if (staged[2]) {
        CR(cudaEventRecord(m->ev_hdone, m->stream));
        CR(cudaStreamWaitEvent(m->d2h, m->ev_hdone, 0));
        CR(cudaMemcpyAsync(arg[2], use[2], sizeof(double), cudaMemcpyDeviceToHost, m->d2h));
    }
    CR(cudaStreamSynchronize(m->d2h));
    CR(cudaStreamSynchronize(m->stream));
    CR(cudaStreamSynchronize(m->h2d));
    return EXA_OK;
}

exa_status exa_jprod(exa_model *m, const double *x, const double *v, double *Jv) {
    if (exa_status e = check_model(m)) return e;
    if (!m->ncon) return EXA_OK;
    CHECK_PTRS(x, v, Jv);
    ExaOut o{};
    o.jac = m->d_jbuf;
    if (exa_status e = launch_eval(m, exa::M_JAC, x, nullptr, 0.0, o)) return e;
    k_spmv_warp<<<grid_of(m->ncon, 256), 256, 0, m->stream>>>(m->d_jrptr, m->d_jrperm, m->d_jbuf, m->d_jcol, v, Jv,
                                                                 (int)m->ncon);
    CR(cudaGetLastError());
    return EXA_OK;
}

exa_status exa_jtprod(exa_model *m, const double *x, const double *w, double *Jtw) {
    if (exa_status e = check_model(m)) return e;
    if (!m->nvar) return EXA_OK;
    CHECK_PTRS(x, Jtw);
    if (m->ncon && !w) return fail(m, EXA_E_INVALID, "NULL w");
    ExaOut o{};
    o.jac = m->d_jbuf;
    if (exa_status e = launch_eval(m, exa::M_JAC, x, nullptr, 0.0, o)) return e;
    k_spmv_warp<<<grid_of(m->nvar, 256), 256, 0, m->stream>>>(m->d_jcolptr_coo, m->d_jperm, m->d_jbuf, m->d_jrow, w,
                                                                 Jtw, (int)m->nvar);
    CR(cudaGetLastError());
    return EXA_OK;
}

exa_status exa_hprod(exa_model *m, const double *x, const double *y, double sigma, const double *v, double *Hv) {
    if (exa_status e = check_model(m)) return e;
    if (!m->nvar) return EXA_OK;
    CHECK_PTRS(x, v, Hv);
    if (m->ncon && !y) return fail(m, EXA_E_INVALID, "NULL y");
    // Hessian CSC values first (duplicates summed once), then the product over unique entries
    if (m->nnzh)
        if (exa_status e = exa_hess_csc(m, x, y, sigma, m->d_hcscbuf)) return e;
    k_hprod_csc<<<grid_of(m->nvar, 256), 256, 0, m->stream>>>(m->d_hcolptr, m->d_hrowval, m->d_hcscbuf, m->d_hcsr_ptr,
                                                               m->d_hcsr_perm, m->d_hcolof, v, Hv, (int)m->nvar);
    CR(cudaGetLastError());
    return EXA_OK;
}

exa_status exa_debug_hold_step(exa_model *m, int32_t member) {
    if (exa_status e = check_model(m)) return e;
    if (!m->fused_step) return fail(m, EXA_E_INVALID, "the model was not created with EXA_FLAG_FUSED_STEP");
    if (member < 0 || member >= m->nb) return fail(m, EXA_E_INVALID, "no such batch member");
    m->step_hold = member;
    return EXA_OK;
}

exa_status exa_check_status(exa_model *m) {
    if (exa_status e = check_model(m)) return e;
    CR(cudaStreamSynchronize(m->stream));
    int st = 0;
    CR(cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CR(cudaMemset(m->d_status, 0, sizeof(int)));
    if (st & 1) return fail(m, EXA_E_BOUNDS, "device bounds check failed");
    if (st & 2) return fail(m, EXA_E_TIMEOUT, "device wait timed out");
    return EXA_OK;
}

exa_status exa_compile_check(const exa_model_desc *desc, const exa_options *opt, char *log, size_t loglen) {
    exa_model tmp;
    exa_status s = EXA_OK;
    if (!desc || desc->n_patterns < 0 || (desc->n_patterns > 0 && !desc->patterns)) {
        s = fail(&tmp, EXA_E_INVALID, "NULL or malformed descriptor");
    } else {
        exa_options o{};
        if (opt) o = *opt;
        s = load_patterns(*desc, &tmp);
        const exa_model_desc *d1[1] = {desc};
        if (s == EXA_OK) s = build_groups(&tmp, d1, 1, (o.flags & EXA_FLAG_NO_FUSE) == 0);
        if (s == EXA_OK) {
            exa::CodegenOptions cg;
            cg.precision = o.precision;
            cg.block = o.block_threads ? o.block_threads : 128;
            cg.bounds_check = (o.flags & EXA_FLAG_BOUNDS_CHECK) != 0;
            cg.by_pattern = (o.flags & EXA_FLAG_UPFRONT) == 0;
            cg.min_blocks = o.min_blocks;
            cg.prefetch = (o.flags & EXA_FLAG_PF_GATHERS) ? 2 : (o.flags & EXA_FLAG_PF_COLUMNS) ? 1 : 0;
            cg.lanes = (o.flags & EXA_FLAG_LANES2) ? 2 : 1;
            cg.lazy_loads = (o.flags & EXA_FLAG_LAZY_LOADS) != 0;
            cg.stage = (o.flags & EXA_FLAG_STAGE_SMEM) != 0;
            cg.fused_step = (o.flags & EXA_FLAG_FUSED_STEP) != 0;
            std::string gerr;
            std::string src = exa::generate_source(tmp.pats, tmp.groups, cg, &gerr);
            if (!gerr.empty()) s = fail(&tmp, EXA_E_INTERNAL, gerr);
            else {
                if (getenv("EXA_DUMP_SOURCE")) {
                    FILE *fp = fopen(getenv("EXA_DUMP_SOURCE"), "w");
                    if (fp) { fputs(src.c_str(), fp); fclose(fp); }
                }
                std::vector<char> cubin;
                s = nvrtc_compile(&tmp, src, cubin);
            }
        }
    }
    if (log && loglen) {
        std::snprintf(log, loglen, "%s", tmp.err.c_str());
    }
    return s;
}

exa_status exa_stat(const exa_model *m, const char *key, double *value) {
    if (!m || !key || !value) return EXA_E_INVALID;
    std::string k(key);
    if (k == "nvrtc_ms") *value = m->nvrtc_ms;
    else if (k == "create_ms") *value = m->create_ms;
    else if (k == "eval_regs") *value = m->regs[exa::M_ALL];
    else if (k == "eval_regs_hess") *value = m->regs[exa::M_HESS];
    else if (k == "eval_regs_jac") *value = m->regs[exa::M_JAC];
    else if (k == "eval_block") *value = m->block;
    else if (k == "eval_persist") *value = m->persist;
    else if (k == "eval_min_blocks") *value = m->min_blocks;
    else if (k == "eval_grid") *value = m->grid[exa::M_ALL];
    else if (k == "tune_ms") *value = m->tune_ms;
    else if (k == "eval_split") *value = m->split_all;
    else if (k == "csc_direct") *value = m->csc_direct;
    else if (k == "hess_compressed") *value = m->use_hcomp;
    else if (k == "eval_chunks") *value = m->nchunks;
    else if (k == "eval_upfront") *value = !m->by_pattern;
    else if (k == "eval_prefetch") *value = m->prefetch;
    else if (k == "eval_lanes") *value = m->lanes;
    else if (k == "eval_lazy") *value = m->lazy_loads;
    else if (k == "eval_stage") *value = m->stage;
    else if (k == "eval_fused_step") *value = m->fused_step;
    else if (k == "eval_kernel_ms") {  // evaluation kernel(s) of the latest exa_eval_all step
        float ms = -1.0f;
        if (!m->ev_k_valid || cudaEventSynchronize(m->ev_k1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, m->ev_k0, m->ev_k1) != cudaSuccess)
            ms = -1.0f;
        *value = ms;
    }
    else if (k == "eval_kernel_kind") {  // which generated kernel(s) the exa_eval_all step with every output runs
        // 0 exa_all, 1 exa_all_b (COO and compressed Hessian sums), 2 exa_first + exa_hess,
        // 3 exa_first + exa_hess_b
        const bool hc = m->use_hcomp && !(m->csc_direct && m->nnzh_csc == m->nnzh);
        *value = (m->split_all ? 2 : 0) + (hc ? 1 : 0);
    }
    else if (k == "eval_dsmem") *value = m->dsmem[exa::M_ALL];
    else if (k == "eval_wave_pct") *value = m->wave_pct;
    else if (k == "graph_kernels") *value = m->graph_kernels;
    else if (k == "grad_compact") *value = m->grad_compact;
    else if (k == "nnzh_compressed") *value = (double)m->nnzhc;
    else if (k == "eval_tiles") *value = m->ntiles[exa::M_ALL];
    else if (k == "device_bytes") *value = (double)m->device_bytes;
    else if (k == "n_patterns") *value = (double)m->pats.size();
    else if (k == "batch_members") *value = m->nb;
    else return EXA_E_INVALID;
    return EXA_OK;
}

}  // extern "C"
