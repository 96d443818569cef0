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
#define EXA_MAXF 16
#define EXA_DEVICE_STRUCTS                                                                          \
    struct ExaPM {                /* one (batch member, pattern) pair */                            \
        const void *f[16];        /* device data columns of this member's pattern */               \
        long long n_inst;         /* instances */                                                   \
        long long xoff;           /* first variable of the member */                                \
        long long nvar_m;         /* variables of the member */                                     \
        long long rbase;          /* CON: row of instance 0; AUG: first row of target block */      \
        long long rlimit;         /* AUG: rows of the target block */                               \
        long long jbase;          /* first Jacobian COO slot of this block */                       \
        long long hbase;          /* first Hessian COO slot of this block */                        \
        long long gbase;          /* first gradient-buffer slot (objective patterns) */             \
        long long abase;          /* first augmentation-buffer entry (augmentation patterns) */     \
        long long poff;           /* first parameter of the member */                               \
        long long npar_m;         /* parameters of the member */                                    \
        long long ic[8];          /* index constants that differ between batch members */           \
        double fc[8];             /* value constants that differ between batch members */           \
        int pat;                  /* pattern id */                                                  \
        int member;               /* batch member */                                                \
    };                                                                                              \
    struct ExaTile {              /* BLOCK consecutive instances of one (member, pattern) */        \
        int pm;                                                                                     \
        int begin;                                                                                  \
        int oslot;                /* objective tiles: index of this tile's partial sum; else -1 */  \
    };                                                                                              \
    struct ExaOut {                                                                                 \
        double *obj_part;         /* one objective partial sum per tile */                          \
        double *c;                /* constraint base values, indexed by global row */               \
        double *abuf;             /* augmentation terms */                                          \
        double *gbuf;             /* objective gradient slots */                                    \
        double *jac;              /* Jacobian COO values */                                         \
        double *hess;             /* Hessian COO values */                                          \
        int *status;              /* device fault word (bounds) */                                  \
    };                                                                                              \
    struct ExaStructOut {                                                                           \
        int *jrow, *jcol, *hrow, *hcol, *gvar, *arow;                                               \
        int *status;                                                                                \
    };

EXA_DEVICE_STRUCTS

namespace exa {

// Generated kernels, one per callback kind: values of objective / constraint patterns, first order
// (gradient slots / Jacobian), second order (Hessian), all of them, all but second order, and the
// structure pass that writes the COO rows and columns.
enum Mode { M_OBJ = 0, M_CON, M_GRAD, M_JAC, M_HESS, M_ALL, M_FIRST, M_STRUCT, M_COUNT };
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
    std::map<int, int> ivary, fvary;
    int nj() const { return (int)jsym.size(); }
    int nh() const { return (int)hpair.size(); }
};

// Validates a pattern (tree shape, opcodes, field types) and computes symbols and slot tables.
// Returns an empty string on success, else the error message.
std::string analyse_pattern(Pattern &p);

// Emits the CUDA C++ source of all generated kernels for the model.
struct CodegenOptions {
    int precision = EXA_FP64;
    int block = 128;
    bool bounds_check = false;
};
std::string generate_source(const std::vector<Pattern> &pats, const CodegenOptions &opt,
                            std::string *err);

extern const char *const kDeviceStructs;

// Symbol id of every Var leaf of the pattern's tree when its index nodes are `ix` (a batch member
// may carry other constants than member 0); -1 for other nodes.
std::vector<int> symbol_partition(const Pattern &p, const std::vector<INode> &ix);

}  // namespace exa
