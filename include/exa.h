/*
 * exa.h -- C ABI of the GB300 derivative-evaluation library for SIMD-form NLPs.
 *
 * Problem class (Eq. (nlp) and Eq. (simd), Sec. 2.1-2.2):
 *     min f(x)  s.t.  gl <= c(x) <= gu,  xl <= x <= xu,
 *     f(x) = sum_l sum_i f_l(x; theta, p_i),
 *     c(x) = [ base rows g_m(x; theta, q_j) ]  +  sum of augmentation terms h_n(x; theta, s_k),
 * where every pattern is one expression tree evaluated over its own data array.  Bounds never
 * enter derivative values and are not part of this interface.
 *
 * The calls follow the solver-facing callbacks of Sec. 2.1 (obj, grad!, cons!, jac_structure!,
 * jac_coord!, hess_structure!, hess_coord!, jprod!, jtprod!, hprod!):
 *   - structure is queried once, values are recomputed per iterate;
 *   - Jacobian and Hessian values are written in the partially compressed COO layout of
 *     Sec. 5.2.2 / 5.3.2: patterns in declaration order, instance k of pattern P owning slots
 *     [o_P + k * step_P, o_P + (k+1) * step_P); only the lower triangle (row >= col) of the
 *     Hessian is stored;
 *   - the CSC calls additionally sum duplicate (row, col) entries into the fully compressed
 *     pattern (the conversion the paper leaves to the solver, Sec. 5.2.2).
 *
 * Conventions for every call below:
 *   - Indices are 0-based (the paper's Julia code is 1-based).
 *   - Array arguments of the evaluation and structure calls are DEVICE pointers on the model's
 *     device, owned by the caller, sized from exa_dims() (exa_eval_all_host also takes host
 *     pointers).  Descriptor arguments of exa_create
 *     are HOST pointers; the library copies what it needs before returning.
 *   - Evaluation calls are stream-ordered and asynchronous on the model's stream (default: the
 *     legacy default stream; see exa_set_stream).  They never synchronize the device and never
 *     allocate device memory, with one exception: exa_eval_all_host, the variant for host
 *     arrays, allocates its staging buffers on first use and returns after synchronizing the
 *     stream.  Inputs must stay valid and unmodified until the enqueued work has run; outputs
 *     are valid once it has run.
 *   - Results do not depend on the launch configuration except through floating-point
 *     summation order (the duplicate sums and the objective reduction are deterministic for a
 *     fixed configuration).
 *   - No exception crosses the ABI.  Every call returns an exa_status; the message of the last
 *     failure is returned by exa_last_error (per model) or exa_create_error (per thread).
 *   - A model is immutable after creation; concurrent calls on different streams are safe when
 *     they use different output buffers and different models, or when they are serialised.
 *     Two calls on one model share its internal work buffers and must not overlap in time.
 */
#ifndef EXA_H
#define EXA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct exa_model exa_model; /* opaque; owned by the library until exa_destroy */

typedef enum {
    EXA_OK = 0,
    EXA_E_INVALID = 1,     /* malformed descriptor or argument (NULL, wrong kind, bad opcode) */
    EXA_E_OOM = 2,         /* device or host allocation failed during exa_create */
    EXA_E_NVRTC = 3,       /* runtime compilation of the generated kernels failed */
    EXA_E_CUDA = 4,        /* a CUDA runtime call failed (message holds the CUDA error) */
    EXA_E_BOUNDS = 5,      /* a resolved variable / parameter / row index is out of range */
    EXA_E_TIMEOUT = 6,     /* a bounded device-side wait expired */
    EXA_E_UNSUPPORTED = 7, /* valid request this build cannot serve (e.g. no sm_103 device) */
    EXA_E_INTERNAL = 8     /* internal consistency check failed */
} exa_status;

typedef enum {
    EXA_FP64 = 0,       /* all pattern arithmetic in FP64 */
    EXA_MIXED_FP32 = 1  /* pattern arithmetic in FP32; FP64 for x loads, trig/exp argument
                           formation and reduction, all cross-instance sums, and outputs */
} exa_precision;

/* ------------------------------------------------------------------ pattern IR opcodes */
/* Value nodes (postorder; children precede parents; the last node is the root). */
enum {
    EXA_V_CONST = 0,  /* fval */
    EXA_V_DATA = 1,   /* data field ival of this instance (int32 fields are converted to double) */
    EXA_V_VAR = 2,    /* x[index expression rooted at inode a] */
    EXA_V_PARAM = 3,  /* theta[index expression rooted at inode a] (no derivatives) */
    EXA_V_NEG = 10, EXA_V_ABS2, EXA_V_INV, EXA_V_EXP, EXA_V_LOG, EXA_V_SIN, EXA_V_COS,
    EXA_V_SQRT, EXA_V_TAN, EXA_V_TANH, EXA_V_ATAN,
    EXA_V_POWI = 21,  /* child a raised to the integer ival */
    EXA_V_SINH = 22, EXA_V_COSH, EXA_V_ASIN, EXA_V_ACOS, EXA_V_LOG1P, EXA_V_EXPM1, EXA_V_LOG2,
    EXA_V_LOG10, EXA_V_EXP2,  /* = 30; registered functions of Sec. 7.1.4 beyond the basic set */
    EXA_V_ADD = 40, EXA_V_SUB, EXA_V_MUL, EXA_V_DIV,
    EXA_V_POW = 44,   /* a ^ b for real b; a must be positive where derivatives are taken */
    EXA_V_ATAN2 = 45, /* atan2(a, b) */
    EXA_V_HYPOT = 46  /* hypot(a, b) */
};
/* Integer index nodes (postorder within the pattern's inode array), 64-bit arithmetic. */
enum {
    EXA_I_CONST = 0,  /* ival */
    EXA_I_FIELD = 1,  /* int32 data field ival of this instance */
    EXA_I_INST = 2,   /* the instance number k = 0 .. n_inst-1 */
    EXA_I_ADD = 10, EXA_I_SUB = 11, EXA_I_MUL = 12
};
enum { EXA_OBJ = 0, EXA_CON = 1, EXA_AUG = 2 };           /* pattern kinds (Sec. 3.3) */
enum { EXA_FIELD_I32 = 0, EXA_FIELD_F64 = 1 };            /* data column types */

typedef struct { int32_t op, a, b, pad; int64_t ival; double fval; } exa_vnode;
typedef struct { int32_t op, a, b, pad; int64_t ival; } exa_inode;
typedef struct { int32_t type, pad; const void *data; } exa_field; /* host column, n_inst long */

/* One pattern (SIMDFunction plus its data, Sec. 3.4):
 *   EXA_OBJ: contributes its value to f; gradient slots; Hessian weighted by sigma.
 *   EXA_CON: instance k defines row row_base + k (row_limit = n_inst rows); Hessian weighted by
 *            y[row].
 *   EXA_AUG: instance k adds its value to row row_base + idx(k), idx = the index expression at
 *            inode row_root, which must lie in [0, row_limit) (the target block's rows);
 *            Jacobian entries on that row; Hessian weighted by y[that row].
 * Two Var leaves are the same symbol iff their index subtrees are structurally identical. */
typedef struct {
    int32_t kind;
    int32_t n_fields;
    int64_t n_inst;
    int64_t row_base;
    int64_t row_limit;
    int32_t row_root;
    int32_t n_vnodes;
    int32_t n_inodes;
    int32_t pad;
    const exa_vnode *vnodes;
    const exa_inode *inodes;
    const exa_field *fields;
} exa_pattern_desc;

typedef struct {
    int64_t nvar, ncon, npar;
    const double *theta;              /* npar host values */
    int32_t n_patterns;
    int32_t pad;
    const exa_pattern_desc *patterns; /* in declaration order: fixes the COO block order */
} exa_model_desc;

/* Creation options.  Zero-initialised options are valid (FP64, automatic launch shape). */
typedef struct {
    int32_t precision;     /* exa_precision */
    int32_t device;        /* CUDA device ordinal */
    int32_t block_threads; /* threads per CTA of the evaluation kernels (multiple of 32, <= 1024);
                              0 = chosen by the autotuner among 64 / 128 / 256 */
    int32_t flags;         /* EXA_FLAG_* */
    int32_t grid_factor;   /* evaluation grid: 0 = chosen by the autotuner (one CTA per tile when
                              tuning is off), -1 = one CTA per tile, n > 0 = persistent grid of n
                              waves of resident CTAs looping over the tiles */
    int32_t min_blocks;    /* launch-bounds minimum resident CTAs per SM of the evaluation kernels
                              (caps their registers), 0..32; 0 = none, or chosen by the autotuner */
    int32_t chunks;        /* exa_eval_all over this many contiguous groups of batch members, the
                              reductions of one group overlapping the evaluation of the next,
                              0..16; 0 = chosen by the autotuner (1 when tuning is off) */
    int32_t wave_pct;      /* 1..99: the evaluation kernels run as a persistent grid of this
                              percentage of one wave of resident CTAs, leaving SM room for the
                              reductions of the previous member chunk to run beside them;
                              0 = per grid_factor, or chosen by the autotuner */
} exa_options;

enum {
    EXA_FLAG_BOUNDS_CHECK = 1, /* every gather index is checked on the device; a violation makes
                                  the next exa_check_status return EXA_E_BOUNDS */
    EXA_FLAG_NO_TUNE = 2,      /* skip the launch-shape autotuner at creation */
    EXA_FLAG_NO_FUSE = 4,      /* evaluate every pattern in its own thread (no fused groups) */
    EXA_FLAG_NO_GRAPH = 8,     /* exa_eval_all launches its kernels directly instead of replaying a
                                  cached CUDA graph */
    /* The next four (and the two prefetch flags below) fix choices the autotuner otherwise makes (they apply as given when tuning is
     * off: EXA_FLAG_NO_TUNE, or block_threads / grid_factor set).  exa_stat reports the choices. */
    EXA_FLAG_SPLIT = 16,       /* exa_eval_all evaluates first and second order in two kernels */
    EXA_FLAG_CSC_SCATTER = 32, /* a duplicate-free CSC is scattered by the evaluation kernel instead
                                  of gathered from the COO values by a permutation kernel */
    EXA_FLAG_NO_HCOMP = 64,    /* the Hessian CSC is summed from the COO slots instead of from the
                                  per-instance sums of the slots of a fused group that share an entry */
    EXA_FLAG_UPFRONT = 128,    /* the generated code computes all of a fused group's arithmetic
                                  before its first output, instead of each pattern's arithmetic right
                                  before that pattern's outputs (the default, which keeps fewer
                                  values live) */
    EXA_FLAG_PF_COLUMNS = 256, /* the evaluation kernels prefetch into L2 the data columns of the
                                  tile two tile-steps ahead (a tile-step: a CTA's next tile in a
                                  persistent grid, else one wave of resident CTAs) */
    EXA_FLAG_PF_GATHERS = 512, /* as EXA_FLAG_PF_COLUMNS, and every thread also prefetches the x and
                                  y lines its instance of the next tile-step gathers */
    EXA_FLAG_LANES2 = 1024,    /* two warp sets per instance: the warps of a CTA form two sets that
                                  evaluate the same instances, each a contiguous subset of a fused
                                  group's patterns (fewer registers per thread); block_threads must
                                  be a multiple of 64; excludes the prefetch flags.  The kernels
                                  that form the compressed Hessian sums keep one set */
    EXA_FLAG_LAZY_LOADS = 2048, /* with the default emission order: each pattern's inputs (x values,
                                  f64 data, parameters, multipliers) are loaded just before the
                                  arithmetic of the pattern preceding it, not all at the top of the
                                  fused group (fewer values live); excludes EXA_FLAG_UPFRONT */
    EXA_FLAG_STAGE_SMEM = 4096, /* staging depth 1: the tile loop copies the inputs of the CTA's next
                                  tile (data columns, x values indexed by the instance alone,
                                  constraint multipliers) into shared memory with cp.async while the
                                  current tile computes from a second buffer; gathers through data
                                  fields still load from global memory.  Excludes EXA_FLAG_LANES2 and
                                  the prefetch flags; ignored with EXA_FLAG_BOUNDS_CHECK */
    EXA_FLAG_HOST_SERIAL = 8192, /* exa_eval_all_host on a batch: no member-chunk pipeline (inputs,
                                  graph, outputs one after another on the model stream) */
    EXA_FLAG_FUSED_STEP = 16384 /* exa_eval_all with the Hessian runs one persistent kernel whose
                                  CTAs take evaluation tiles and reductions (Jacobian and Hessian CSC,
                                  gradient, constraint augmentations) from one work queue; a
                                  member's reductions wait (bounded; EXA_E_TIMEOUT from
                                  exa_check_status if the bound is hit) for that member's tiles, so
                                  on a batch they overlap the evaluation of later members.  FP64
                                  models only; excludes EXA_FLAG_STAGE_SMEM, EXA_FLAG_LANES2 and the
                                  prefetch flags; with member chunks or EXA_FLAG_SPLIT the plain
                                  graph is used.  Not chosen by the autotuner */
};

/* Validate the descriptor (Sec. 3.4 SIMDFunction), lower every pattern to generated device
 * code and compile it with NVRTC for sm_103a, copy the data columns to the device, run the
 * device structure pass (COO rows/cols of every slot, Sec. 5.3.1) and the device sorts that fix
 * the COO->CSC permutation and the gradient/augmentation segment pointers.  Synchronizes the
 * device.  On failure *out is NULL and exa_create_error() holds the message. */
exa_status exa_create(const exa_model_desc *desc, const exa_options *opt, exa_model **out);

/* Batch of nb models with identical pattern trees (same IR, Sec. 7.4.3) but their own data and
 * sizes.  The batch behaves as one model whose x, y, c, and every COO array are the members'
 * arrays concatenated in member order; member b's slice equals what exa_create on member b alone
 * produces.  Offsets of each member: exa_batch_offsets. */
exa_status exa_create_batch(const exa_model_desc *const *descs, int32_t nb, const exa_options *opt,
                            exa_model **out);

void exa_destroy(exa_model *m); /* synchronizes the model's stream, frees device memory */

const char *exa_last_error(const exa_model *m); /* never NULL; "" if no error */
const char *exa_create_error(void);             /* message of this thread's last failed create */

/* Problem dimensions.  nnzj/nnzh count COO slots (duplicates included); *_csc count the
 * distinct (row, col) entries.  Any output pointer may be NULL. */
exa_status exa_dims(const exa_model *m, int64_t *nvar, int64_t *ncon, int64_t *nnzj, int64_t *nnzh,
                    int64_t *nnzj_csc, int64_t *nnzh_csc);

/* For batch models: per member b (nb + 1 entries each, prefix form) the first variable, row,
 * Jacobian slot and Hessian slot of member b.  Any pointer may be NULL.  A plain model has nb=1. */
exa_status exa_batch_offsets(const exa_model *m, int32_t *nb, int64_t *xoff, int64_t *coff,
                             int64_t *joff, int64_t *hoff);

/* Replace the parameter values theta (host array of npar doubles, all batch members' parameters
 * concatenated in member order), as the paper's parameter update does without rebuilding the model
 * (Sec. 2.1: theta is held fixed during a solve and may change between solves).  The copy is
 * ordered on the model's stream and the call synchronizes that stream, so the host array may be
 * reused once the call returns. */
exa_status exa_set_theta(exa_model *m, const double *theta, int64_t npar);

/* Stream (a cudaStream_t) on which every later call on this model enqueues its work. */
exa_status exa_set_stream(exa_model *m, void *stream);

/* ------------------------------------------------------------------ callbacks (Sec. 2.1) */
/* f[0] = f(x).  f: one device double.  Objective terms are reduced in FP64 in two stages (every
 * CTA sums the terms of all its tiles into one partial, then one ordered sum of the partials),
 * Sec. 7.2.3. */
exa_status exa_obj(exa_model *m, const double *x, double *f);

/* f[0] = f(x), like exa_obj, but without the scratch buffer that exa_create allocates: the
 * per-CTA partial sums go to a fixed static device array of 65536 doubles (512 KiB) that every GPU
 * which loads the library holds until the process exits.  For callers that cannot allocate device
 * memory (their memory belongs to another allocator, or they run where cudaMalloc is not allowed);
 * this call allocates nothing.  The paper has no counterpart; it is an addition of this library.
 *   - Limit: at most 65536 partial sums, one per CTA of the objective kernel's launch
 *     (EXA_E_UNSUPPORTED beyond, with the count in the message; f is then left untouched).  With
 *     one CTA per tile that is one per objective tile, counted per batch member and fused pattern
 *     group as ceil(objective instances / block), block being the launch shape's threads per CTA
 *     (exa_stat "eval_block"; 64 to 256 when tuned): 8,388,608 instances of one pattern at block
 *     128, fewer when a batch has many members or groups; a persistent grid (exa_stat
 *     "eval_grid") launches fewer CTAs.
 *   - Every call looks up the array's address on the model's device (a CUDA runtime query, no
 *     allocation).  The first call on a device may also load the library's device code there:
 *     make that first call before any stream capture.
 *   - Every call shares the one array: calls that overlap on the same GPU race.  Nothing needs
 *     clearing between calls; each call overwrites every partial it reads. */
exa_status exa_obj_noalloc(exa_model *m, const double *x, double *f);

/* g[nvar] = grad f(x): each objective instance writes its own gradient slots, then a gather
 * segmented sum per variable produces g (Sec. 7.2.3, no atomics). */
exa_status exa_grad(exa_model *m, const double *x, double *g);

/* c[ncon] = base rows plus augmentation terms (Sec. 3.3, 7.2.3). */
exa_status exa_cons(exa_model *m, const double *x, double *c);

/* COO structure: rows[nnzj], cols[nnzj] (device int32). */
exa_status exa_jac_structure(const exa_model *m, int32_t *rows, int32_t *cols);
/* COO values vals[nnzj] of the constraint Jacobian at x. */
exa_status exa_jac_coord(exa_model *m, const double *x, double *vals);

/* Lower-triangle COO structure (row >= col), rows[nnzh], cols[nnzh]. */
exa_status exa_hess_structure(const exa_model *m, int32_t *rows, int32_t *cols);
/* COO values vals[nnzh] of sigma * Hess f(x) + sum_r y[r] Hess c_r(x).  A slot pairing two
 * different symbols that resolve to the same variable holds twice the mixed partial, so the
 * symmetric expansion of the COO sum is the Hessian. */
exa_status exa_hess_coord(exa_model *m, const double *x, const double *y, double sigma,
                          double *vals);

/* CSC structure of the Jacobian (ncon x nvar) and of the Hessian's lower triangle (nvar x nvar):
 * colptr[nvar+1], rowval[nnz*_csc] (rows ascending within a column), coo2csc[nnz*]: the CSC
 * position of every COO slot.  Built on the device at creation by a stable sort of (col, row). */
exa_status exa_jac_csc_structure(const exa_model *m, int32_t *colptr, int32_t *rowval,
                                 int32_t *coo2csc);
exa_status exa_hess_csc_structure(const exa_model *m, int32_t *colptr, int32_t *rowval,
                                  int32_t *coo2csc);
/* CSC values: the COO values of each (row, col) summed in ascending COO order. */
exa_status exa_jac_csc(exa_model *m, const double *x, double *vals_csc);
exa_status exa_hess_csc(exa_model *m, const double *x, const double *y, double sigma,
                        double *vals_csc);

/* Everything in one pass over all patterns.  Any output may be NULL (not computed).
 * jac/hess are COO values; jac_csc/hess_csc CSC values.  y and sigma are read only when hess or
 * hess_csc is requested.  The launches are replayed from a CUDA graph cached per argument tuple
 * (4 tuples kept; the first call with a new tuple captures it); when the model's stream is being
 * captured by the caller, the launches are recorded into that capture instead. */
exa_status exa_eval_all(exa_model *m, const double *x, const double *y, double sigma, double *f,
                        double *g, double *c, double *jac, double *hess, double *jac_csc,
                        double *hess_csc);

/* exa_eval_all for callers whose arrays live in host memory: every argument (sizes as in
 * exa_eval_all) may be host memory, page-locked or pageable, or device memory.  Host inputs are
 * copied into device buffers the library owns (allocated on first use), the exa_eval_all graph is
 * replayed on the model stream, host outputs are copied back, and the call returns when they are
 * in host memory (the stream is synchronized).  Device arguments are used in place.  For a batch
 * of two or more members the call is pipelined over up to 8 member chunks of about equal
 * nonzeros: the chunks' inputs are copied in on a stream of their own, chunk k is evaluated
 * (directly launched, not from the graph) once its inputs are in, and its outputs (every output
 * of a member is a contiguous range) are copied back on another stream as soon as its reductions
 * have run, overlapping the copies of later chunks; the objective follows the last chunk.  Single
 * models, EXA_FLAG_HOST_SERIAL, and calls while the model stream is being captured copy all inputs,
 * replay the graph and then copy the outputs back one after another on the model stream.
 * Page-locked host buffers (cudaHostAlloc / cudaHostRegister) are copied at full link speed. */
exa_status exa_eval_all_host(exa_model *m, const double *x, const double *y, double sigma,
                             double *f, double *g, double *c, double *jac, double *hess,
                             double *jac_csc, double *hess_csc);

/* Products at x (NLPModels jprod!/jtprod!/hprod!): Jv[ncon] = J(x) v, Jtw[nvar] = J(x)^T w,
 * Hv[nvar] = (sigma Hess f + sum y_r Hess c_r)(x) v with the Hessian's full symmetric action. */
exa_status exa_jprod(exa_model *m, const double *x, const double *v, double *Jv);
exa_status exa_jtprod(exa_model *m, const double *x, const double *w, double *Jtw);
exa_status exa_hprod(exa_model *m, const double *x, const double *y, double sigma,
                     const double *v, double *Hv);

/* Synchronizes the model's stream and reports device-side faults recorded by bounded waits or
 * bounds checks since the last call (EXA_E_BOUNDS, EXA_E_TIMEOUT), clearing them. */
exa_status exa_check_status(exa_model *m);

/* Failure injection for tests of the fused step's bounded wait (EXA_FLAG_FUSED_STEP models only):
 * the next exa_eval_all call starts `member`'s tile counter one below zero, so that it ends one
 * short of the member's tiles; that member's reductions poll for a short bound (4096 polls), give
 * up and run on what is there, the kernel finishes, and exa_check_status then reports
 * EXA_E_TIMEOUT.  One call only (launched directly, not from the cached graph); later calls are
 * normal.  EXA_E_INVALID for other models or a member out of range. */
exa_status exa_debug_hold_step(exa_model *m, int32_t member);

/* Validate the descriptor, generate the kernels and compile them with NVRTC for sm_103a without
 * touching any device (usable on a host without a GPU).  With the environment variable
 * EXA_DUMP_SOURCE set to a file name, this call and exa_create write the generated CUDA source
 * there (for reading the code a model compiles to).  On failure the message (NVRTC log
 * included) is copied, NUL-terminated, into log[0 .. loglen-1] when log is not NULL. */
exa_status exa_compile_check(const exa_model_desc *desc, const exa_options *opt, char *log,
                             size_t loglen);

/* Named statistics (host values): "nvrtc_ms", "create_ms", "tune_ms", "eval_regs", "eval_block",
 * "eval_regs_jac", "eval_regs_hess", "eval_tiles", "eval_grid", "eval_persist", "eval_min_blocks",
 * "eval_split", "eval_chunks", "eval_upfront", "eval_prefetch", "eval_wave_pct", "eval_lanes", "eval_lazy",
 * "eval_stage", "eval_dsmem", "eval_fused_step", "graph_kernels", "csc_direct",
 * "hess_compressed", "nnzh_compressed", "grad_compact", "device_bytes", "n_patterns", "batch_members".
 * "eval_kernel_ms": milliseconds between CUDA events recorded on the model stream right before and
 * right after the evaluation kernel(s) of the latest exa_eval_all call (also inside its cached
 * graphs; member chunks: the first chunk's launch to the last chunk's); waits for the second event;
 * -1 when no call has recorded them.  "eval_kernel_kind": the generated kernel(s) an exa_eval_all
 * call with every output runs: 0 exa_all, 1 exa_all_b (COO and compressed Hessian sums),
 * 2 exa_first + exa_hess, 3 exa_first + exa_hess_b.
 * Unknown key: EXA_E_INVALID. */
exa_status exa_stat(const exa_model *m, const char *key, double *value);

#ifdef __cplusplus
}
#endif
#endif /* EXA_H */
