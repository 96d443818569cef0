// exa_internal.h -- internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/exa.h"

// Device-visible descriptors.  The same text is compiled into the host library and, via the
// stringised copy kDeviceStructs, into every NVRTC-generated module, so both sides agree on the
// layout by construction.
#define EXA_MAXF 16  /* data columns per fused group */
#define EXA_MAXG 16  /* patterns per fused group */
#define EXA_DEVICE_STRUCTS                                                                          \
    struct ExaPM {                /* one (batch member, fused pattern group) pair */               \
        const void *f[16];        /* device data columns of the group (shared columns once) */     \
        const float *f32[16];     /* mixed mode: FP32 copies of the f64 columns */                  \
        long long n_inst;         /* instances (equal for every pattern of the group) */           \
        long long xoff;           /* first variable of the member */                                \
        long long nvar_m;         /* variables of the member */                                     \
        long long poff;           /* first parameter of the member */                               \
        long long npar_m;         /* parameters of the member */                                    \
        long long ic[16];         /* index constants that differ between batch members */           \
        double fc[16];            /* value constants that differ between batch members */           \
        long long rbase[16];      /* per pattern: CON row of instance 0 / AUG first target row */   \
        long long rlimit[16];     /* per pattern: AUG rows of the target block */                   \
        long long jbase[16];      /* per pattern: first Jacobian COO slot */                        \
        long long hbase[16];      /* per pattern: first Hessian COO slot */                         \
        long long gbase[16];      /* per pattern: first gradient-buffer slot */                     \
        long long abase[16];      /* per pattern: first augmentation-buffer entry */                \
        long long hcbase;         /* first slot of the group's compressed Hessian sums */           \
        int grp;                  /* group id */                                                    \
        int member;               /* batch member */                                                \
    };                                                                                              \
    struct ExaTile {              /* BLOCK consecutive instances of one (member, group) */          \
        int pm;                                                                                     \
        int begin;                                                                                  \
    };                                                                                              \
    struct ExaOut {                                                                                 \
        double *obj_part;         /* one objective partial sum per CTA of the launch */             \
        double *c;                /* constraint base values, indexed by global row */               \
        double *abuf;             /* augmentation terms */                                          \
        double *gbuf;             /* objective gradient slots */                                    \
        double *jac;              /* Jacobian COO values */                                         \
        double *hess;             /* Hessian COO values */                                          \
        double *jcsc;             /* if set: Jacobian CSC values written directly (no duplicates) */\
        const int *jmap;          /* Jacobian COO slot -> CSC position */                           \
        double *hcsc;             /* if set: Hessian CSC values written directly (no duplicates) */ \
        const int *hmap;          /* Hessian COO slot -> CSC position */                            \
        double *hcomp;            /* if set: per-instance sums of the group's equal Hessian pairs */\
        int *status;              /* device fault word (bounds) */                                  \
    };                                                                                              \
    struct ExaStructOut {                                                                           \
        int *jrow, *jcol, *hrow, *hcol, *gvar, *arow, *hcrow, *hccol;                               \
        int *status;                                                                                \
    };                                                                                              \
    struct ExaTask {              /* one item of the fused step's work queue */                     \
        int kind;                 /* 0: evaluation tile p0; k > 0: reduction r[k - 1] over [p0,p1) */\
        int member;               /* batch member the tile belongs to / the reduction waits for */  \
        int p0, p1;                                                                                 \
    };                                                                                              \
    struct ExaRed {               /* one reduction of the fused step */                             \
        int how;                  /* -1 off; 0 dst[p] = src[perm[p]]; segment sums over           */\
                                  /* perm[ptr[s] .. ptr[s+1]): 1 dst[s] from the first entry,     */\
                                  /* 2 dst[s] from 0.0, 3 dst[rows[s]] plus the segment            */\
        const int *ptr, *perm, *rows;                                                               \
        const double *src;                                                                          \
        double *dst;                                                                                \
    };                                                                                              \
    struct ExaStep {                                                                                \
        int *ctr;                 /* ctr[0]: next queue item; ctr[1 + b]: finished tiles of b */     \
        const int *need;          /* evaluation tiles of each member */                             \
        const ExaTask *items;     /* the queue */                                                   \
        int nitems;                                                                                 \
        int spin_limit;           /* bound on a reduction's wait for its member's tiles */          \
        ExaRed r[4];              /* Jacobian CSC, Hessian CSC, gradient, constraint augmentations */\
    };

EXA_DEVICE_STRUCTS

namespace exa {

// Generated kernels, one per callback kind: values of objective / constraint patterns, first order
// (gradient slots / Jacobian), second order (Hessian), all of them, all but second order, and the
// structure pass that writes the COO rows and columns.  The Hessian-producing kinds come in three
// compile-time variants: COO slots (M_HESS, M_ALL), the group-compressed sums used for the CSC
// (..._C), or both (..._B).
enum Mode { M_OBJ = 0, M_CON, M_GRAD, M_JAC, M_HESS, M_ALL, M_FIRST, M_STRUCT,
            M_HESS_C, M_HESS_B, M_ALL_C, M_ALL_B, M_COUNT };
inline bool mode_hess(int m) { return m == M_HESS || m == M_ALL || m >= M_HESS_C; }
inline bool mode_all(int m) { return m == M_ALL || m == M_ALL_C || m == M_ALL_B; }
inline bool mode_hess_coo(int m) { return m == M_HESS || m == M_ALL || m == M_HESS_B || m == M_ALL_B; }
inline bool mode_hess_comp(int m) { return m >= M_HESS_C; }
extern const char *const kModeName[M_COUNT];

struct VNode { int op, a, b; long long iv; double fv; };
struct INode { int op, a, b; long long iv; };

struct Pattern {
    int kind = 0;
    long long n_inst = 0, row_base = 0, row_limit = 0;
    int row_root = -1;
    std::vector<VNode> v;
    std::vector<INode> ix;
    std::vector<int> ftype;
    // structure (filled by analyse)
    int nsym = 0;
    std::vector<int> sym_of;    // per value node: symbol of a VAR leaf, else -1
    std::vector<int> sym_root;  // per symbol: its index-expression root
    std::vector<int> jsym;      // first-order slot -> symbol
    std::vector<std::pair<int, int>> hpair;  // Hessian slot -> symbol pair (as first emitted)
    // constants that differ between batch members: node index -> slot in ExaPM::ic / ExaPM::fc
    // (slots are numbered per fused group)
    std::map<int, int> ivary, fvary;
    int nj() const { return (int)jsym.size(); }
    int nh() const { return (int)hpair.size(); }
};

// Patterns evaluated by one thread per instance (equal instance counts in every batch member).
struct Group {
    std::vector<int> pats;                  // pattern ids in declaration order
    std::vector<int> ftype;                 // per group data column
    std::vector<std::vector<int>> field;    // [position][pattern field] -> group column
    std::vector<std::vector<int>> sym;      // [position][pattern symbol] -> group symbol
    std::vector<std::pair<int, int>> sym_root;  // group symbol -> (position, index root) defining it
    int nic = 0, nfc = 0;                   // member-varying constant slots in use
    // compressed Hessian: slots of the group's patterns over the same pair of group symbols (the
    // same (row, col) for every instance), summed per instance; each entry lists (position, slot)
    std::vector<std::vector<std::pair<int, int>>> hc;
    std::vector<std::pair<int, int>> hc_sym;  // group symbol pair of each compressed slot
};

// Unifies the symbols of a group's patterns: equal index expressions (columns compared as group
// columns, member-varying constants as slots) are one group symbol.
void finalize_group(Group &g, const std::vector<Pattern> &pats);

// Validates a pattern (tree shape, opcodes, field types) and computes symbols and slot tables.
// Returns an empty string on success, else the error message.
std::string analyse_pattern(Pattern &p);

// Emits the CUDA C++ source of all generated kernels for the model.
struct CodegenOptions {
    int precision = EXA_FP64;
    int block = 128;
    int min_blocks = 0;  // __launch_bounds__ minimum resident CTAs per SM (0: not given)
    bool bounds_check = false;
    // emit each pattern's arithmetic just before its outputs (shorter live ranges) instead of all
    // of a group's arithmetic before the first output
    bool by_pattern = true;
    // with by_pattern: load each pattern's inputs (x values, f64 data, parameters, multipliers) just
    // before the arithmetic of the pattern preceding it, instead of all at the top of the group
    bool lazy_loads = false;
    // L2 prefetch of later tiles' inputs in the tile loop: 0 none; 1 the data columns of the tile
    // 2 x pfd ahead (one bulk prefetch per column); 2 also the x and y lines the tile pfd ahead
    // gathers (pfd: a kernel argument, the CTA's next tile in a persistent grid, else one wave)
    int prefetch = 0;
    // Warp sets per instance: with 2, the warps of a CTA form two sets that evaluate the same
    // instances of a tile, each its own contiguous subset of a fused group's patterns (fewer values
    // live per thread; shared subexpressions recomputed by both).  Kinds that form the compressed
    // Hessian sums, and groups with a single active pattern, keep one set.  Excludes prefetch.
    int lanes = 1;
    // Shared-memory staging of inputs (1: on): the persistent tile loop copies the data columns,
    // the x values indexed by the instance alone and the constraint multipliers of the CTA's next
    // tile into a second buffer of per-thread slots (cp.async) while the current tile computes from
    // the first.  Excludes prefetch, warp sets and bounds checking.
    int stage = 0;
    // Fused step kernels (exa_step, exa_step_b): the evaluation tiles of the M_ALL / M_ALL_B kernel
    // and the step's reductions taken from one work queue (ExaStep).  Excludes staging, prefetch
    // and warp sets.
    bool fused_step = false;
};
// The warp sets of group g in kernel kind `mode` (positions in g.pats per set, in order): one set
// with every active pattern, or `lanes` contiguous subsets of about equal outputs.
std::vector<std::vector<int>> group_sets(const std::vector<Pattern> &pats, const Group &g, Mode mode, int lanes);
// dsmem (optional, M_COUNT entries): the dynamic shared memory each kernel kind needs, in bytes.
std::string generate_source(const std::vector<Pattern> &pats, const std::vector<Group> &groups,
                            const CodegenOptions &opt, std::string *err, int *dsmem = nullptr);
bool pattern_in_mode(const Pattern &p, Mode m);

extern const char *const kDeviceStructs;

// Symbol id of every Var leaf of the pattern's tree when its index nodes are `ix` (a batch member
// may carry other constants than member 0); -1 for other nodes.
std::vector<int> symbol_partition(const Pattern &p, const std::vector<INode> &ix);

}  // namespace exa
