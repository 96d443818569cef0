/*
 * exa_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the derivative-evaluation
 * path of the SIMD-form NLP (Eq. (simd), Sec. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline call this file.  It shares no code with the GPU library: it has its own reader of the
 * flat pattern IR, its own structure rule and its own AD.
 *
 * What it computes, per model:
 *   f(x)         = sum over objective patterns and their instances of the pattern value (Eq. (simd)).
 *   grad f       = dense gradient; duplicate contributions summed in ascending buffer order.
 *   c(x)         = base constraint values plus augmentation terms (Sec. 3.3), ascending order.
 *   J (COO)      = Jacobian values in the partially compressed COO layout (Sec. 5.2.2, 5.3.2).
 *   H (COO)      = lower triangle of  sigma * Hess f + sum_r y_r Hess c_r  (Sec. 2.1 callbacks).
 *   CSC          = stable sort of (col, row, COO index), duplicates summed in ascending COO order.
 *   Jv, J^T w, Hv from the COO entries.
 *
 * How:
 *   - Structure (Sec. 5.2.1-5.2.2): a probe walks each pattern tree once in the order a reverse
 *     pass visits it and records symbolic variable references; a compressor maps every raw visit
 *     to the first unique occurrence.  Symbols are Var leaves with structurally equal index
 *     expressions.  First-order visits are the Var leaves in pre-order, left to right.  The
 *     second-order probe follows the reverse-over-reverse rule of Sec. 5.1.3: a node passes a
 *     "second adjoint may be nonzero" flag to each child (set if the parent's flag is set or the
 *     op's own second partial for that child is not identically zero); a leaf with the flag set
 *     emits its diagonal pair; a binary node, after both children, emits every (leaf of child 1,
 *     leaf of child 2) pair if its flag is set or its mixed second partial is not identically zero.
 *     Pairs are deduplicated as unordered symbol pairs.  Global entries are (max, min) of the
 *     resolved indices (Sec. 5.2.2: lower triangle only).
 *   - Values: per instance, the postorder node array is the tape.  A forward sweep stores each
 *     node's value and local first and second partials; one reverse sweep gives the gradient over
 *     symbols; the local Hessian is built column by column with forward-over-reverse (tangent
 *     sweep with seed e_s, then a reverse sweep of adjoints and adjoint tangents).  This is a
 *     different AD mode from the GPU's generated code (reverse over reverse), by design.
 *   - A Hessian entry of two different symbols that resolve to the same variable at run time lands
 *     on the diagonal; it is stored doubled so that the symmetric expansion of the COO sum equals
 *     the Hessian over variables.
 *   - Every local Hessian entry that the structure rule leaves out must be exactly zero; if not,
 *     evaluation fails with ORC_E_STRUCT (a structure-bug detector).
 *
 * Self-check helpers: complex-valued evaluation of the objective and constraints (for complex-step
 * first derivatives) and a complex-valued first-order AD gradient of the Lagrangian (for a
 * complex-step Hessian that uses only first-derivative rules).
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_INVALID 1
#define ORC_E_OOM 2
#define ORC_E_BOUNDS 3
#define ORC_E_STRUCT 4

/* opcodes of the flat IR */
enum { OV_CONST = 0, OV_DATA = 1, OV_VAR = 2, OV_PARAM = 3,
       OV_NEG = 10, OV_ABS2, OV_INV, OV_EXP, OV_LOG, OV_SIN, OV_COS, OV_SQRT, OV_TAN, OV_TANH,
       OV_ATAN, OV_POWI, OV_SINH, OV_COSH, OV_ASIN, OV_ACOS, OV_LOG1P, OV_EXPM1, OV_LOG2,
       OV_LOG10, OV_EXP2,
       OV_ADD = 40, OV_SUB, OV_MUL, OV_DIV, OV_POW, OV_ATAN2, OV_HYPOT };
enum { OI_CONST = 0, OI_FIELD = 1, OI_INST = 2, OI_ADD = 10, OI_SUB = 11, OI_MUL = 12 };
enum { OK_OBJ = 0, OK_CON = 1, OK_AUG = 2 };

typedef struct {
    int kind;
    int64_t n_inst, row_base, row_limit;
    int row_root;
    int nv; int *vop, *va, *vb; int64_t *vi; double *vf;
    int ni; int *iop, *ia, *ib; int64_t *ii;
    int nf; int *ftype; const void **fptr;
    /* structure, filled by analyse() */
    int nsym;
    int *sym_of;          /* per value node: symbol id of a VAR node, else -1 */
    int *sym_root;        /* per symbol: index-expression root */
    int nraw1, *raw1, *comp1;           /* first-order raw visits (symbols) and their slots */
    int nj, *jsym;                      /* first-order slot -> symbol */
    int nraw2, *raw2a, *raw2b, *comp2;  /* second-order raw visits and their slots */
    int nh, *ha, *hb;                   /* Hessian slot -> symbol pair */
    int64_t o_jac, o_hess, o_grad;      /* block offsets */
} opat;

typedef struct {
    int64_t nvar, ncon, npar;
    double *theta;
    int np, cap;
    opat *p;
    int64_t nnzj, nnzh, nnzg;
    int finalized;
    /* CSC */
    int64_t nnzj_csc, nnzh_csc;
    int32_t *jrow, *jcol, *hrow, *hcol;        /* COO structure */
    int32_t *j_colptr, *j_rowval, *j_coo2csc;
    int32_t *h_colptr, *h_rowval, *h_coo2csc;
    char err[256];
} orc_model;

/* ------------------------------------------------------------------ small helpers */
static void *xmalloc(size_t n) { return malloc(n ? n : 1); }
static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

static int set_err(orc_model *m, int code, const char *msg) {
    snprintf(m->err, sizeof m->err, "%s", msg);
    return code;
}

static int is_unary(int op) { return op >= OV_NEG && op <= OV_EXP2; }
static int is_binary(int op) { return op >= OV_ADD && op <= OV_HYPOT; }

/* ------------------------------------------------------------------ construction */
orc_model *orc_new(int64_t nvar, int64_t ncon, int64_t npar, const double *theta) {
    orc_model *m = (orc_model *)xcalloc(1, sizeof(orc_model));
    m->nvar = nvar; m->ncon = ncon; m->npar = npar;
    m->theta = (double *)xmalloc(sizeof(double) * (size_t)npar);
    if (npar) memcpy(m->theta, theta, sizeof(double) * (size_t)npar);
    return m;
}

const char *orc_error(const orc_model *m) { return m->err; }

static void *dup(const void *src, size_t bytes) {
    void *d = xmalloc(bytes);
    if (bytes) memcpy(d, src, bytes);
    return d;
}

int orc_add_pattern(orc_model *m, int kind, int64_t n_inst, int64_t row_base, int64_t row_limit,
                    int row_root, int nv, const int *vop, const int *va, const int *vb,
                    const int64_t *vi, const double *vf, int ni, const int *iop, const int *ia,
                    const int *ib, const int64_t *ii, int nf, const int *ftype,
                    const void *const *fptr) {
    if (m->finalized) return set_err(m, ORC_E_INVALID, "model already finalized");
    if (m->np == m->cap) {
        m->cap = m->cap ? 2 * m->cap : 8;
        m->p = (opat *)realloc(m->p, sizeof(opat) * (size_t)m->cap);
    }
    opat *p = &m->p[m->np++];
    memset(p, 0, sizeof *p);
    p->kind = kind; p->n_inst = n_inst; p->row_base = row_base; p->row_limit = row_limit;
    p->row_root = row_root;
    p->nv = nv;
    p->vop = (int *)dup(vop, sizeof(int) * (size_t)nv);
    p->va = (int *)dup(va, sizeof(int) * (size_t)nv);
    p->vb = (int *)dup(vb, sizeof(int) * (size_t)nv);
    p->vi = (int64_t *)dup(vi, sizeof(int64_t) * (size_t)nv);
    p->vf = (double *)dup(vf, sizeof(double) * (size_t)nv);
    p->ni = ni;
    p->iop = (int *)dup(iop, sizeof(int) * (size_t)ni);
    p->ia = (int *)dup(ia, sizeof(int) * (size_t)ni);
    p->ib = (int *)dup(ib, sizeof(int) * (size_t)ni);
    p->ii = (int64_t *)dup(ii, sizeof(int64_t) * (size_t)ni);
    p->nf = nf;
    p->ftype = (int *)dup(ftype, sizeof(int) * (size_t)nf);
    p->fptr = (const void **)dup(fptr, sizeof(void *) * (size_t)nf);
    return ORC_OK;
}

/* ------------------------------------------------------------------ index expressions */
static int idx_equal(const opat *p, int r1, int r2) {
    if (r1 == r2) return 1;
    if (p->iop[r1] != p->iop[r2]) return 0;
    switch (p->iop[r1]) {
    case OI_CONST: case OI_FIELD: return p->ii[r1] == p->ii[r2];
    case OI_INST: return 1;
    default: return idx_equal(p, p->ia[r1], p->ia[r2]) && idx_equal(p, p->ib[r1], p->ib[r2]);
    }
}

static int64_t idx_eval(const opat *p, int r, int64_t k) {
    switch (p->iop[r]) {
    case OI_CONST: return p->ii[r];
    case OI_FIELD: return (int64_t)((const int32_t *)p->fptr[p->ii[r]])[k];
    case OI_INST: return k;
    case OI_ADD: return idx_eval(p, p->ia[r], k) + idx_eval(p, p->ib[r], k);
    case OI_SUB: return idx_eval(p, p->ia[r], k) - idx_eval(p, p->ib[r], k);
    default: return idx_eval(p, p->ia[r], k) * idx_eval(p, p->ib[r], k);
    }
}

static double data_val(const opat *p, int64_t f, int64_t k) {
    if (p->ftype[f] == 0) return (double)((const int32_t *)p->fptr[f])[k];
    return ((const double *)p->fptr[f])[k];
}

/* ------------------------------------------------------------------ validation */
static int check_idx_tree(orc_model *m, const opat *p, int r, int limit) {
    if (r < 0 || r >= limit) return set_err(m, ORC_E_INVALID, "index node reference out of order");
    int op = p->iop[r];
    if (op == OI_CONST || op == OI_INST) return ORC_OK;
    if (op == OI_FIELD) {
        if (p->ii[r] < 0 || p->ii[r] >= p->nf || p->ftype[p->ii[r]] != 0)
            return set_err(m, ORC_E_INVALID, "index expression reads a missing or non-int32 field");
        return ORC_OK;
    }
    if (op != OI_ADD && op != OI_SUB && op != OI_MUL)
        return set_err(m, ORC_E_INVALID, "unknown index opcode");
    int e = check_idx_tree(m, p, p->ia[r], r);
    if (e) return e;
    return check_idx_tree(m, p, p->ib[r], r);
}

static int validate_pattern(orc_model *m, const opat *p) {
    if (p->kind < OK_OBJ || p->kind > OK_AUG) return set_err(m, ORC_E_INVALID, "bad pattern kind");
    if (p->n_inst < 0) return set_err(m, ORC_E_INVALID, "negative instance count");
    if (p->nv < 1) return set_err(m, ORC_E_INVALID, "empty pattern tree");
    for (int f = 0; f < p->nf; f++)
        if (p->ftype[f] != 0 && p->ftype[f] != 1) return set_err(m, ORC_E_INVALID, "bad field type");
    for (int n = 0; n < p->nv; n++) {
        int op = p->vop[n];
        if (op == OV_CONST) continue;
        if (op == OV_DATA) {
            if (p->vi[n] < 0 || p->vi[n] >= p->nf) return set_err(m, ORC_E_INVALID, "data field out of range");
            continue;
        }
        if (op == OV_VAR || op == OV_PARAM) {
            int e = check_idx_tree(m, p, p->va[n], p->ni);
            if (e) return e;
            continue;
        }
        if (is_unary(op)) {
            if (p->va[n] < 0 || p->va[n] >= n) return set_err(m, ORC_E_INVALID, "child must precede parent");
            continue;
        }
        if (is_binary(op)) {
            if (p->va[n] < 0 || p->va[n] >= n || p->vb[n] < 0 || p->vb[n] >= n)
                return set_err(m, ORC_E_INVALID, "child must precede parent");
            continue;
        }
        return set_err(m, ORC_E_INVALID, "unknown value opcode");
    }
    if (p->kind == OK_AUG) {
        int e = check_idx_tree(m, p, p->row_root, p->ni);
        if (e) return e;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ structure rule */
/* Is the op's second partial with respect to its child(ren) identically zero?  (Sec. 7.2.2)
 * which: 1 = d2/du1^2, 2 = d2/du2^2, 3 = d2/du1du2. */
static int second_nonzero(const opat *p, int n, int which) {
    int op = p->vop[n];
    switch (op) {
    case OV_NEG: return 0;
    case OV_POWI: return !(p->vi[n] == 0 || p->vi[n] == 1);
    case OV_ADD: case OV_SUB: return 0;
    case OV_MUL: return which == 3;
    case OV_DIV: return which != 1;
    case OV_POW: return 1;
    default: return 1; /* abs2, inv, exp, log, sin, cos, sqrt, tan, tanh, atan */
    }
}

static int has_var(const opat *p, int n) {
    int op = p->vop[n];
    if (op == OV_VAR) return 1;
    if (op == OV_CONST || op == OV_DATA || op == OV_PARAM) return 0;
    if (is_unary(op)) return has_var(p, p->va[n]);
    return has_var(p, p->va[n]) || has_var(p, p->vb[n]);
}

typedef struct { int *a, *b; int n, cap; } pairlist;
static void pl_push(pairlist *l, int a, int b) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 16;
        l->a = (int *)realloc(l->a, sizeof(int) * (size_t)l->cap);
        l->b = (int *)realloc(l->b, sizeof(int) * (size_t)l->cap);
    }
    l->a[l->n] = a; l->b[l->n] = b; l->n++;
}

/* first-order probe: Var leaves in pre-order, left to right */
static void probe1(const opat *p, int n, pairlist *raw) {
    int op = p->vop[n];
    if (op == OV_VAR) { pl_push(raw, p->sym_of[n], 0); return; }
    if (is_unary(op)) { probe1(p, p->va[n], raw); return; }
    if (is_binary(op)) { probe1(p, p->va[n], raw); probe1(p, p->vb[n], raw); }
}

static void leaves(const opat *p, int n, pairlist *out) { probe1(p, n, out); }

/* second-order probe (reverse over reverse, structural) */
static void probe2(const opat *p, int n, int z2, pairlist *raw) {
    int op = p->vop[n];
    if (op == OV_VAR) { if (z2) pl_push(raw, p->sym_of[n], p->sym_of[n]); return; }
    if (op == OV_CONST || op == OV_DATA || op == OV_PARAM) return;
    if (is_unary(op)) { probe2(p, p->va[n], z2 || second_nonzero(p, n, 1), raw); return; }
    int h1 = has_var(p, p->va[n]), h2 = has_var(p, p->vb[n]);
    if (h1) probe2(p, p->va[n], z2 || second_nonzero(p, n, 1), raw);
    if (h2) probe2(p, p->vb[n], z2 || second_nonzero(p, n, 2), raw);
    if (h1 && h2 && (z2 || second_nonzero(p, n, 3))) {
        pairlist l1 = {0}, l2 = {0};
        leaves(p, p->va[n], &l1);
        leaves(p, p->vb[n], &l2);
        for (int i = 0; i < l1.n; i++)
            for (int j = 0; j < l2.n; j++) pl_push(raw, l1.a[i], l2.a[j]);
        free(l1.a); free(l1.b); free(l2.a); free(l2.b);
    }
}

static int analyse(orc_model *m, opat *p) {
    /* symbols */
    p->sym_of = (int *)xmalloc(sizeof(int) * (size_t)p->nv);
    p->sym_root = (int *)xmalloc(sizeof(int) * (size_t)p->nv);
    p->nsym = 0;
    for (int n = 0; n < p->nv; n++) p->sym_of[n] = -1;
    /* symbol ids in order of first pre-order occurrence: collect VAR nodes in pre-order */
    pairlist pre = {0};
    {
        /* iterative pre-order with an explicit stack */
        int *st = (int *)xmalloc(sizeof(int) * (size_t)(p->nv + 1));
        int sp = 0;
        st[sp++] = p->nv - 1;
        while (sp) {
            int n = st[--sp];
            int op = p->vop[n];
            if (op == OV_VAR) pl_push(&pre, n, 0);
            else if (is_unary(op)) st[sp++] = p->va[n];
            else if (is_binary(op)) { st[sp++] = p->vb[n]; st[sp++] = p->va[n]; }
        }
        free(st);
    }
    for (int i = 0; i < pre.n; i++) {
        int n = pre.a[i], s = -1;
        for (int t = 0; t < p->nsym; t++)
            if (idx_equal(p, p->sym_root[t], p->va[n])) { s = t; break; }
        if (s < 0) { s = p->nsym++; p->sym_root[s] = p->va[n]; }
        p->sym_of[n] = s;
    }
    free(pre.a); free(pre.b);

    /* first-order compressor */
    pairlist r1 = {0};
    probe1(p, p->nv - 1, &r1);
    p->nraw1 = r1.n;
    p->raw1 = (int *)xmalloc(sizeof(int) * (size_t)r1.n);
    p->comp1 = (int *)xmalloc(sizeof(int) * (size_t)r1.n);
    p->jsym = (int *)xmalloc(sizeof(int) * (size_t)(p->nsym + 1));
    p->nj = 0;
    for (int i = 0; i < r1.n; i++) {
        int s = r1.a[i], slot = -1;
        p->raw1[i] = s;
        for (int j = 0; j < p->nj; j++) if (p->jsym[j] == s) { slot = j; break; }
        if (slot < 0) { slot = p->nj++; p->jsym[slot] = s; }
        p->comp1[i] = slot;
    }
    free(r1.a); free(r1.b);

    /* second-order compressor: unique unordered symbol pairs */
    pairlist r2 = {0};
    probe2(p, p->nv - 1, 0, &r2);
    p->nraw2 = r2.n;
    p->raw2a = (int *)xmalloc(sizeof(int) * (size_t)r2.n);
    p->raw2b = (int *)xmalloc(sizeof(int) * (size_t)r2.n);
    p->comp2 = (int *)xmalloc(sizeof(int) * (size_t)r2.n);
    p->ha = (int *)xmalloc(sizeof(int) * (size_t)r2.n);
    p->hb = (int *)xmalloc(sizeof(int) * (size_t)r2.n);
    p->nh = 0;
    for (int i = 0; i < r2.n; i++) {
        int a = r2.a[i], b = r2.b[i], slot = -1;
        p->raw2a[i] = a; p->raw2b[i] = b;
        for (int j = 0; j < p->nh; j++)
            if ((p->ha[j] == a && p->hb[j] == b) || (p->ha[j] == b && p->hb[j] == a)) { slot = j; break; }
        if (slot < 0) { slot = p->nh++; p->ha[slot] = a; p->hb[slot] = b; }
        p->comp2[i] = slot;
    }
    free(r2.a); free(r2.b);
    (void)m;
    return ORC_OK;
}

/* ------------------------------------------------------------------ structure per instance */
static int64_t pattern_row(const opat *p, int64_t k) {
    if (p->kind == OK_CON) return p->row_base + k;
    if (p->kind == OK_AUG) return p->row_base + idx_eval(p, p->row_root, k);
    return -1;
}

static int cmp_key3(const void *x, const void *y) {
    const int64_t *a = (const int64_t *)x, *b = (const int64_t *)y;
    for (int i = 0; i < 3; i++) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

/* CSC of a COO pattern: sort (col, row, coo index) -- the index makes the order stable. */
static void build_csc(int64_t nnz, int64_t ncol, const int32_t *row, const int32_t *col,
                      int64_t *nnz_csc, int32_t **colptr, int32_t **rowval, int32_t **coo2csc) {
    int64_t *keys = (int64_t *)xmalloc(sizeof(int64_t) * 3 * (size_t)nnz);
    for (int64_t q = 0; q < nnz; q++) {
        keys[3 * q] = col[q]; keys[3 * q + 1] = row[q]; keys[3 * q + 2] = q;
    }
    qsort(keys, (size_t)nnz, sizeof(int64_t) * 3, cmp_key3);
    *colptr = (int32_t *)xcalloc((size_t)ncol + 1, sizeof(int32_t));
    *rowval = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)nnz);
    *coo2csc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)nnz);
    int64_t u = -1;
    for (int64_t i = 0; i < nnz; i++) {
        int64_t c = keys[3 * i], r = keys[3 * i + 1], q = keys[3 * i + 2];
        if (i == 0 || c != keys[3 * (i - 1)] || r != keys[3 * (i - 1) + 1]) {
            u++;
            (*rowval)[u] = (int32_t)r;
            (*colptr)[c + 1]++;
        }
        (*coo2csc)[q] = (int32_t)u;
    }
    for (int64_t c = 0; c < ncol; c++) (*colptr)[c + 1] += (*colptr)[c];
    *nnz_csc = u + 1;
    free(keys);
}

int orc_finalize(orc_model *m) {
    if (m->finalized) return ORC_OK;
    if (m->nvar < 0 || m->ncon < 0 || m->npar < 0) return set_err(m, ORC_E_INVALID, "negative size");
    if (m->nvar >= INT32_MAX || m->ncon >= INT32_MAX) return set_err(m, ORC_E_INVALID, "size too large");
    for (int i = 0; i < m->np; i++) {
        int e = validate_pattern(m, &m->p[i]);
        if (e) return e;
        analyse(m, &m->p[i]);
    }
    /* offsets in declaration order */
    int64_t oj = 0, oh = 0, og = 0;
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        p->o_hess = oh; oh += p->n_inst * p->nh;
        if (p->kind == OK_OBJ) { p->o_grad = og; og += p->n_inst * p->nj; p->o_jac = -1; }
        else { p->o_jac = oj; oj += p->n_inst * p->nj; p->o_grad = -1; }
    }
    m->nnzj = oj; m->nnzh = oh; m->nnzg = og;
    if (oj >= INT32_MAX || oh >= INT32_MAX) return set_err(m, ORC_E_INVALID, "too many nonzeros");
    /* resolve structure and validate indices */
    m->jrow = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)oj);
    m->jcol = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)oj);
    m->hrow = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)oh);
    m->hcol = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)oh);
    int64_t *sidx = (int64_t *)xmalloc(sizeof(int64_t) * 64);
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        if (p->nsym > 64) { free(sidx); sidx = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)p->nsym); }
        for (int64_t k = 0; k < p->n_inst; k++) {
            for (int s = 0; s < p->nsym; s++) {
                sidx[s] = idx_eval(p, p->sym_root[s], k);
                if (sidx[s] < 0 || sidx[s] >= m->nvar) { free(sidx); return set_err(m, ORC_E_BOUNDS, "variable index out of range"); }
            }
            for (int n = 0; n < p->nv; n++)
                if (p->vop[n] == OV_PARAM) {
                    int64_t t = idx_eval(p, p->va[n], k);
                    if (t < 0 || t >= m->npar) { free(sidx); return set_err(m, ORC_E_BOUNDS, "parameter index out of range"); }
                }
            int64_t row = pattern_row(p, k);
            if (p->kind == OK_AUG) {
                int64_t local = row - p->row_base;
                if (local < 0 || local >= p->row_limit) { free(sidx); return set_err(m, ORC_E_BOUNDS, "augmentation row out of its block"); }
            }
            if (p->kind != OK_OBJ && (row < 0 || row >= m->ncon)) { free(sidx); return set_err(m, ORC_E_BOUNDS, "constraint row out of range"); }
            if (p->kind != OK_OBJ)
                for (int j = 0; j < p->nj; j++) {
                    int64_t q = p->o_jac + k * p->nj + j;
                    m->jrow[q] = (int32_t)row;
                    m->jcol[q] = (int32_t)sidx[p->jsym[j]];
                }
            for (int j = 0; j < p->nh; j++) {
                int64_t q = p->o_hess + k * p->nh + j;
                int64_t a = sidx[p->ha[j]], b = sidx[p->hb[j]];
                m->hrow[q] = (int32_t)(a > b ? a : b);
                m->hcol[q] = (int32_t)(a > b ? b : a);
            }
        }
    }
    free(sidx);
    build_csc(oj, m->nvar, m->jrow, m->jcol, &m->nnzj_csc, &m->j_colptr, &m->j_rowval, &m->j_coo2csc);
    build_csc(oh, m->nvar, m->hrow, m->hcol, &m->nnzh_csc, &m->h_colptr, &m->h_rowval, &m->h_coo2csc);
    m->finalized = 1;
    return ORC_OK;
}

void orc_dims(const orc_model *m, int64_t *out) {
    out[0] = m->nvar; out[1] = m->ncon; out[2] = m->nnzj; out[3] = m->nnzh;
    out[4] = m->nnzj_csc; out[5] = m->nnzh_csc; out[6] = m->nnzg;
}

/* per-pattern structural constants: [nsym, nj (o1step), nh (o2step), nraw1, nraw2] */
void orc_pattern_info(const orc_model *m, int i, int64_t *out) {
    const opat *p = &m->p[i];
    out[0] = p->nsym; out[1] = p->nj; out[2] = p->nh; out[3] = p->nraw1; out[4] = p->nraw2;
}
/* compressor maps, 1-based as printed in Sec. 5.2.2 */
void orc_pattern_comp(const orc_model *m, int i, int32_t *comp1, int32_t *comp2) {
    const opat *p = &m->p[i];
    for (int r = 0; r < p->nraw1; r++) comp1[r] = p->comp1[r] + 1;
    for (int r = 0; r < p->nraw2; r++) comp2[r] = p->comp2[r] + 1;
}

void orc_jac_structure(const orc_model *m, int32_t *rows, int32_t *cols) {
    memcpy(rows, m->jrow, sizeof(int32_t) * (size_t)m->nnzj);
    memcpy(cols, m->jcol, sizeof(int32_t) * (size_t)m->nnzj);
}
void orc_hess_structure(const orc_model *m, int32_t *rows, int32_t *cols) {
    memcpy(rows, m->hrow, sizeof(int32_t) * (size_t)m->nnzh);
    memcpy(cols, m->hcol, sizeof(int32_t) * (size_t)m->nnzh);
}
void orc_jac_csc_structure(const orc_model *m, int32_t *colptr, int32_t *rowval, int32_t *coo2csc) {
    memcpy(colptr, m->j_colptr, sizeof(int32_t) * (size_t)(m->nvar + 1));
    memcpy(rowval, m->j_rowval, sizeof(int32_t) * (size_t)m->nnzj_csc);
    memcpy(coo2csc, m->j_coo2csc, sizeof(int32_t) * (size_t)m->nnzj);
}
void orc_hess_csc_structure(const orc_model *m, int32_t *colptr, int32_t *rowval, int32_t *coo2csc) {
    memcpy(colptr, m->h_colptr, sizeof(int32_t) * (size_t)(m->nvar + 1));
    memcpy(rowval, m->h_rowval, sizeof(int32_t) * (size_t)m->nnzh_csc);
    memcpy(coo2csc, m->h_coo2csc, sizeof(int32_t) * (size_t)m->nnzh);
}

/* ------------------------------------------------------------------ the tape (FP64) */
typedef struct {
    double *val, *d1, *d2, *h11, *h12, *h22;   /* value and local partials per node */
    double *adj, *dot, *adjdot;                /* reverse / tangent work */
    double *grad;                              /* per symbol */
    double *hess;                              /* nsym x nsym, column-major */
    int64_t *sidx;
    int cap, scap;
} tape;

static void tape_reserve(tape *t, int nv, int nsym) {
    if (nv > t->cap) {
        t->cap = nv;
        double **arrs[] = {&t->val, &t->d1, &t->d2, &t->h11, &t->h12, &t->h22, &t->adj, &t->dot, &t->adjdot};
        for (int i = 0; i < 9; i++) { free(*arrs[i]); *arrs[i] = (double *)xmalloc(sizeof(double) * (size_t)nv); }
    }
    if (nsym > t->scap) {
        t->scap = nsym;
        free(t->grad); free(t->hess); free(t->sidx);
        t->grad = (double *)xmalloc(sizeof(double) * (size_t)nsym);
        t->hess = (double *)xmalloc(sizeof(double) * (size_t)nsym * (size_t)nsym);
        t->sidx = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nsym);
    }
}
static void tape_free(tape *t) {
    double *arrs[] = {t->val, t->d1, t->d2, t->h11, t->h12, t->h22, t->adj, t->dot, t->adjdot, t->grad, t->hess};
    for (int i = 0; i < 11; i++) free(arrs[i]);
    free(t->sidx);
}

static double ipow(double u, int64_t n) {
    /* u^n for integer n by repeated multiplication of |n| factors, then reciprocal if n < 0 */
    double r = 1.0;
    int64_t a = n < 0 ? -n : n;
    for (int64_t i = 0; i < a; i++) r *= u;
    return n < 0 ? 1.0 / r : r;
}

/* Forward sweep: value, first and second local partials of every node (Sec. 5.1.1, 5.1.3). */
static void forward(const orc_model *m, const opat *p, int64_t k, const double *x, tape *t) {
    for (int n = 0; n < p->nv; n++) {
        int op = p->vop[n];
        double v = 0, d1 = 0, d2 = 0, h11 = 0, h12 = 0, h22 = 0;
        double u = 0, w = 0;
        if (is_unary(op)) u = t->val[p->va[n]];
        if (is_binary(op)) { u = t->val[p->va[n]]; w = t->val[p->vb[n]]; }
        switch (op) {
        case OV_CONST: v = p->vf[n]; break;
        case OV_DATA: v = data_val(p, p->vi[n], k); break;
        case OV_VAR: v = x[idx_eval(p, p->va[n], k)]; break;
        case OV_PARAM: v = m->theta[idx_eval(p, p->va[n], k)]; break;
        case OV_NEG: v = -u; d1 = -1; break;
        case OV_ABS2: v = u * u; d1 = 2 * u; h11 = 2; break;
        case OV_INV: v = 1 / u; d1 = -1 / (u * u); h11 = 2 / (u * u * u); break;
        case OV_EXP: v = exp(u); d1 = v; h11 = v; break;
        case OV_LOG: v = log(u); d1 = 1 / u; h11 = -1 / (u * u); break;
        case OV_SIN: v = sin(u); d1 = cos(u); h11 = -v; break;
        case OV_COS: v = cos(u); d1 = -sin(u); h11 = -v; break;
        case OV_SQRT: v = sqrt(u); d1 = 0.5 / v; h11 = -0.25 / (u * v); break;
        case OV_TAN: { double c = cos(u); v = tan(u); d1 = 1 / (c * c); h11 = 2 * v * d1; break; }
        case OV_TANH: v = tanh(u); d1 = 1 - v * v; h11 = -2 * v * d1; break;
        case OV_ATAN: v = atan(u); d1 = 1 / (1 + u * u); h11 = -2 * u * d1 * d1; break;
        case OV_POWI: {
            int64_t e = p->vi[n];
            v = ipow(u, e);
            d1 = (double)e * ipow(u, e - 1);
            h11 = (double)e * (double)(e - 1) * ipow(u, e - 2);
            break;
        }
        case OV_SINH: v = sinh(u); d1 = cosh(u); h11 = v; break;
        case OV_COSH: v = cosh(u); d1 = sinh(u); h11 = v; break;
        case OV_ASIN: { double r = 1 / sqrt(1 - u * u); v = asin(u); d1 = r; h11 = u * r * r * r; break; }
        case OV_ACOS: { double r = 1 / sqrt(1 - u * u); v = acos(u); d1 = -r; h11 = -u * r * r * r; break; }
        case OV_LOG1P: v = log1p(u); d1 = 1 / (1 + u); h11 = -d1 * d1; break;
        case OV_EXPM1: v = expm1(u); d1 = exp(u); h11 = d1; break;
        case OV_LOG2: v = log2(u); d1 = 1 / (u * log(2.0)); h11 = -d1 / u; break;
        case OV_LOG10: v = log10(u); d1 = 1 / (u * log(10.0)); h11 = -d1 / u; break;
        case OV_EXP2: v = exp2(u); d1 = v * log(2.0); h11 = d1 * log(2.0); break;
        case OV_ATAN2: {
            double r = u * u + w * w;
            v = atan2(u, w); d1 = w / r; d2 = -u / r;
            h11 = -2 * u * w / (r * r); h12 = (u * u - w * w) / (r * r); h22 = 2 * u * w / (r * r);
            break;
        }
        case OV_HYPOT: {
            v = hypot(u, w); d1 = u / v; d2 = w / v;
            h11 = w * w / (v * v * v); h12 = -u * w / (v * v * v); h22 = u * u / (v * v * v);
            break;
        }
        case OV_ADD: v = u + w; d1 = 1; d2 = 1; break;
        case OV_SUB: v = u - w; d1 = 1; d2 = -1; break;
        case OV_MUL: v = u * w; d1 = w; d2 = u; h12 = 1; break;
        case OV_DIV: v = u / w; d1 = 1 / w; d2 = -u / (w * w); h12 = -1 / (w * w); h22 = 2 * u / (w * w * w); break;
        case OV_POW: {
            v = pow(u, w);
            double lu = log(u);
            d1 = w * pow(u, w - 1);
            d2 = v * lu;
            h11 = w * (w - 1) * pow(u, w - 2);
            h12 = pow(u, w - 1) * (1 + w * lu);
            h22 = v * lu * lu;
            break;
        }
        }
        t->val[n] = v; t->d1[n] = d1; t->d2[n] = d2;
        t->h11[n] = h11; t->h12[n] = h12; t->h22[n] = h22;
    }
}

/* Reverse sweep with seed 1: gradient over symbols (Sec. 5.1.2). */
static void reverse1(const opat *p, tape *t) {
    for (int n = 0; n < p->nv; n++) t->adj[n] = 0;
    for (int s = 0; s < p->nsym; s++) t->grad[s] = 0;
    t->adj[p->nv - 1] = 1;
    for (int n = p->nv - 1; n >= 0; n--) {
        int op = p->vop[n];
        double a = t->adj[n];
        if (op == OV_VAR) t->grad[p->sym_of[n]] += a;
        else if (is_unary(op)) t->adj[p->va[n]] += a * t->d1[n];
        else if (is_binary(op)) {
            t->adj[p->va[n]] += a * t->d1[n];
            t->adj[p->vb[n]] += a * t->d2[n];
        }
    }
}

/* Forward over reverse: column s of the local Hessian over symbols (needs reverse1 first). */
static void hess_column(const opat *p, tape *t, int s) {
    for (int n = 0; n < p->nv; n++) {
        int op = p->vop[n];
        double d = 0;
        if (op == OV_VAR) d = (p->sym_of[n] == s) ? 1 : 0;
        else if (is_unary(op)) d = t->d1[n] * t->dot[p->va[n]];
        else if (is_binary(op)) d = t->d1[n] * t->dot[p->va[n]] + t->d2[n] * t->dot[p->vb[n]];
        t->dot[n] = d;
        t->adjdot[n] = 0;
    }
    double *col = t->hess + (size_t)s * (size_t)p->nsym;
    for (int r = 0; r < p->nsym; r++) col[r] = 0;
    for (int n = p->nv - 1; n >= 0; n--) {
        int op = p->vop[n];
        double ad = t->adjdot[n], a = t->adj[n];
        if (op == OV_VAR) col[p->sym_of[n]] += ad;
        else if (is_unary(op)) {
            int c = p->va[n];
            t->adjdot[c] += ad * t->d1[n] + a * t->h11[n] * t->dot[c];
        } else if (is_binary(op)) {
            int c1 = p->va[n], c2 = p->vb[n];
            double u1 = t->dot[c1], u2 = t->dot[c2];
            t->adjdot[c1] += ad * t->d1[n] + a * (t->h11[n] * u1 + t->h12[n] * u2);
            t->adjdot[c2] += ad * t->d2[n] + a * (t->h12[n] * u1 + t->h22[n] * u2);
        }
    }
}

static void resolve(const opat *p, int64_t k, tape *t) {
    for (int s = 0; s < p->nsym; s++) t->sidx[s] = idx_eval(p, p->sym_root[s], k);
}

static int in_structure(const opat *p, int a, int b) {
    for (int j = 0; j < p->nh; j++)
        if ((p->ha[j] == a && p->hb[j] == b) || (p->ha[j] == b && p->hb[j] == a)) return 1;
    return 0;
}

/* ------------------------------------------------------------------ callbacks */
int orc_obj(orc_model *m, const double *x, double *f) {
    tape t = {0};
    double acc = 0;
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        if (p->kind != OK_OBJ) continue;
        tape_reserve(&t, p->nv, p->nsym);
        for (int64_t k = 0; k < p->n_inst; k++) { forward(m, p, k, x, &t); acc += t.val[p->nv - 1]; }
    }
    tape_free(&t);
    *f = acc;
    return ORC_OK;
}

int orc_cons(orc_model *m, const double *x, double *c) {
    tape t = {0};
    for (int64_t r = 0; r < m->ncon; r++) c[r] = 0;
    for (int pass = 0; pass < 2; pass++)  /* base values first, then augmentations in order */
        for (int i = 0; i < m->np; i++) {
            opat *p = &m->p[i];
            if ((pass == 0 && p->kind != OK_CON) || (pass == 1 && p->kind != OK_AUG)) continue;
            tape_reserve(&t, p->nv, p->nsym);
            for (int64_t k = 0; k < p->n_inst; k++) {
                forward(m, p, k, x, &t);
                int64_t row = pattern_row(p, k);
                if (pass == 0) c[row] = t.val[p->nv - 1];
                else c[row] += t.val[p->nv - 1];
            }
        }
    tape_free(&t);
    return ORC_OK;
}

/* sparse objective gradient buffer (one slot per first-order slot of each objective instance) */
int orc_grad_coo(orc_model *m, const double *x, double *gbuf, int32_t *gvar) {
    tape t = {0};
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        if (p->kind != OK_OBJ) continue;
        tape_reserve(&t, p->nv, p->nsym);
        for (int64_t k = 0; k < p->n_inst; k++) {
            forward(m, p, k, x, &t);
            reverse1(p, &t);
            resolve(p, k, &t);
            for (int j = 0; j < p->nj; j++) {
                int64_t q = p->o_grad + k * p->nj + j;
                if (gbuf) gbuf[q] = t.grad[p->jsym[j]];
                if (gvar) gvar[q] = (int32_t)t.sidx[p->jsym[j]];
            }
        }
    }
    tape_free(&t);
    return ORC_OK;
}

int orc_grad(orc_model *m, const double *x, double *g) {
    double *gbuf = (double *)xmalloc(sizeof(double) * (size_t)m->nnzg);
    int32_t *gvar = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)m->nnzg);
    orc_grad_coo(m, x, gbuf, gvar);
    for (int64_t v = 0; v < m->nvar; v++) g[v] = 0;
    for (int64_t q = 0; q < m->nnzg; q++) g[gvar[q]] += gbuf[q];
    free(gbuf); free(gvar);
    return ORC_OK;
}

int orc_jac_coord(orc_model *m, const double *x, double *vals) {
    tape t = {0};
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        if (p->kind == OK_OBJ) continue;
        tape_reserve(&t, p->nv, p->nsym);
        for (int64_t k = 0; k < p->n_inst; k++) {
            forward(m, p, k, x, &t);
            reverse1(p, &t);
            for (int j = 0; j < p->nj; j++) vals[p->o_jac + k * p->nj + j] = t.grad[p->jsym[j]];
        }
    }
    tape_free(&t);
    return ORC_OK;
}

/* Local Hessian of every instance, weighted by sigma (objective) or y[row] (constraints). */
int orc_hess_coord(orc_model *m, const double *x, const double *y, double sigma, double *vals) {
    tape t = {0};
    int err = ORC_OK;
    for (int i = 0; i < m->np && !err; i++) {
        opat *p = &m->p[i];
        tape_reserve(&t, p->nv, p->nsym);
        for (int64_t k = 0; k < p->n_inst && !err; k++) {
            forward(m, p, k, x, &t);
            reverse1(p, &t);
            for (int s = 0; s < p->nsym; s++) hess_column(p, &t, s);
            resolve(p, k, &t);
            int ns = p->nsym;
            double scale = 0;
            for (int a = 0; a < ns * ns; a++) { double v = fabs(t.hess[a]); if (v > scale) scale = v; }
            for (int a = 0; a < ns; a++)
                for (int b = 0; b < a; b++) {
                    double hab = t.hess[(size_t)b * ns + a], hba = t.hess[(size_t)a * ns + b];
                    if (fabs(hab - hba) > 1e-13 * scale) { err = set_err(m, ORC_E_STRUCT, "local Hessian not symmetric"); }
                }
            for (int a = 0; a < ns && !err; a++)
                for (int b = 0; b <= a; b++)
                    if (!in_structure(p, a, b) && t.hess[(size_t)b * ns + a] != 0.0) {
                        err = set_err(m, ORC_E_STRUCT, "nonzero local Hessian entry outside the structure");
                        break;
                    }
            double w = p->kind == OK_OBJ ? sigma : y[pattern_row(p, k)];
            for (int j = 0; j < p->nh; j++) {
                int a = p->ha[j], b = p->hb[j];
                double h = t.hess[(size_t)b * ns + a];  /* column b, row a */
                if (a != b && t.sidx[a] == t.sidx[b]) h *= 2;  /* off-diagonal pair on the diagonal */
                vals[p->o_hess + k * p->nh + j] = w * h;
            }
        }
    }
    tape_free(&t);
    return err;
}

/* ------------------------------------------------------------------ CSC values */
static void coo_to_csc(int64_t nnz, int64_t nnz_csc, const int32_t *coo2csc, const double *coo, double *csc) {
    for (int64_t p = 0; p < nnz_csc; p++) csc[p] = 0;
    for (int64_t q = 0; q < nnz; q++) csc[coo2csc[q]] += coo[q];  /* ascending COO index */
}
int orc_jac_csc(orc_model *m, const double *x, double *csc) {
    double *coo = (double *)xmalloc(sizeof(double) * (size_t)m->nnzj);
    orc_jac_coord(m, x, coo);
    coo_to_csc(m->nnzj, m->nnzj_csc, m->j_coo2csc, coo, csc);
    free(coo);
    return ORC_OK;
}
int orc_hess_csc(orc_model *m, const double *x, const double *y, double sigma, double *csc) {
    double *coo = (double *)xmalloc(sizeof(double) * (size_t)m->nnzh);
    int e = orc_hess_coord(m, x, y, sigma, coo);
    coo_to_csc(m->nnzh, m->nnzh_csc, m->h_coo2csc, coo, csc);
    free(coo);
    return e;
}

/* ------------------------------------------------------------------ products */
int orc_jprod(orc_model *m, const double *x, const double *v, double *jv) {
    double *coo = (double *)xmalloc(sizeof(double) * (size_t)m->nnzj);
    orc_jac_coord(m, x, coo);
    for (int64_t r = 0; r < m->ncon; r++) jv[r] = 0;
    for (int64_t q = 0; q < m->nnzj; q++) jv[m->jrow[q]] += coo[q] * v[m->jcol[q]];
    free(coo);
    return ORC_OK;
}
int orc_jtprod(orc_model *m, const double *x, const double *w, double *jtw) {
    double *coo = (double *)xmalloc(sizeof(double) * (size_t)m->nnzj);
    orc_jac_coord(m, x, coo);
    for (int64_t c = 0; c < m->nvar; c++) jtw[c] = 0;
    for (int64_t q = 0; q < m->nnzj; q++) jtw[m->jcol[q]] += coo[q] * w[m->jrow[q]];
    free(coo);
    return ORC_OK;
}
int orc_hprod(orc_model *m, const double *x, const double *y, double sigma, const double *v, double *hv) {
    double *coo = (double *)xmalloc(sizeof(double) * (size_t)m->nnzh);
    int e = orc_hess_coord(m, x, y, sigma, coo);
    for (int64_t c = 0; c < m->nvar; c++) hv[c] = 0;
    for (int64_t q = 0; q < m->nnzh; q++) {
        int32_t r = m->hrow[q], c = m->hcol[q];
        hv[r] += coo[q] * v[c];
        if (r != c) hv[c] += coo[q] * v[r];
    }
    free(coo);
    return e;
}

/* ------------------------------------------------------------------ complex-valued checks */
typedef double complex cplx;

static cplx cipow(cplx u, int64_t n) {
    cplx r = 1.0;
    int64_t a = n < 0 ? -n : n;
    for (int64_t i = 0; i < a; i++) r *= u;
    return n < 0 ? 1.0 / r : r;
}

/* atan2 continued analytically off the real axis: atan(a/b) plus the constant that selects the
 * quadrant of the real arguments (constants do not change derivatives); b must not be 0. */
static cplx catan2_(cplx a, cplx b) {
    cplx r = catan(a / b);
    if (creal(b) < 0) r += creal(a) >= 0 ? M_PI : -M_PI;
    return r;
}

/* Value of node n of instance k in complex arithmetic (plain recursive tree walk). */
static cplx ceval(const orc_model *m, const opat *p, int n, int64_t k, const cplx *x) {
    int op = p->vop[n];
    switch (op) {
    case OV_CONST: return p->vf[n];
    case OV_DATA: return data_val(p, p->vi[n], k);
    case OV_VAR: return x[idx_eval(p, p->va[n], k)];
    case OV_PARAM: return m->theta[idx_eval(p, p->va[n], k)];
    default: break;
    }
    cplx u = ceval(m, p, p->va[n], k, x);
    switch (op) {
    case OV_NEG: return -u;
    case OV_ABS2: return u * u;
    case OV_INV: return 1.0 / u;
    case OV_EXP: return cexp(u);
    case OV_LOG: return clog(u);
    case OV_SIN: return csin(u);
    case OV_COS: return ccos(u);
    case OV_SQRT: return csqrt(u);
    case OV_TAN: return ctan(u);
    case OV_TANH: return ctanh(u);
    case OV_ATAN: return catan(u);
    case OV_POWI: return cipow(u, p->vi[n]);
    case OV_SINH: return csinh(u);
    case OV_COSH: return ccosh(u);
    case OV_ASIN: return casin(u);
    case OV_ACOS: return cacos(u);
    case OV_LOG1P: return clog(1.0 + u);
    case OV_EXPM1: return cexp(u) - 1.0;
    case OV_LOG2: return clog(u) / log(2.0);
    case OV_LOG10: return clog(u) / log(10.0);
    case OV_EXP2: return cexp(u * log(2.0));
    default: break;
    }
    cplx w = ceval(m, p, p->vb[n], k, x);
    switch (op) {
    case OV_ADD: return u + w;
    case OV_SUB: return u - w;
    case OV_MUL: return u * w;
    case OV_DIV: return u / w;
    case OV_ATAN2: return catan2_(u, w);
    case OV_HYPOT: return csqrt(u * u + w * w);
    default: return cexp(w * clog(u));
    }
}

static cplx *to_cplx(int64_t n, const double *re, const double *im) {
    cplx *z = (cplx *)xmalloc(sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; i++) z[i] = re[i] + I * (im ? im[i] : 0.0);
    return z;
}

int orc_obj_complex(orc_model *m, const double *xr, const double *xi, double *fr, double *fi) {
    cplx *x = to_cplx(m->nvar, xr, xi), acc = 0;
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        if (p->kind != OK_OBJ) continue;
        for (int64_t k = 0; k < p->n_inst; k++) acc += ceval(m, p, p->nv - 1, k, x);
    }
    *fr = creal(acc); *fi = cimag(acc);
    free(x);
    return ORC_OK;
}

int orc_cons_complex(orc_model *m, const double *xr, const double *xi, double *cr, double *ci) {
    cplx *x = to_cplx(m->nvar, xr, xi);
    cplx *c = (cplx *)xcalloc((size_t)m->ncon, sizeof(cplx));
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        if (p->kind == OK_OBJ) continue;
        for (int64_t k = 0; k < p->n_inst; k++) c[pattern_row(p, k)] += ceval(m, p, p->nv - 1, k, x);
    }
    for (int64_t r = 0; r < m->ncon; r++) { cr[r] = creal(c[r]); ci[r] = cimag(c[r]); }
    free(x); free(c);
    return ORC_OK;
}

/* First-order AD (forward values and first partials, then one reverse sweep) in complex
 * arithmetic; gives grad of  sigma f + y^T c  at complex x.  Its imaginary part over the step
 * is a Hessian column that depends only on first-derivative rules. */
int orc_lag_grad_complex(orc_model *m, const double *xr, const double *xi, const double *y,
                         double sigma, double *gr, double *gi) {
    cplx *x = to_cplx(m->nvar, xr, xi);
    cplx *g = (cplx *)xcalloc((size_t)m->nvar, sizeof(cplx));
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        cplx *val = (cplx *)xmalloc(sizeof(cplx) * (size_t)p->nv);
        cplx *d1 = (cplx *)xmalloc(sizeof(cplx) * (size_t)p->nv);
        cplx *d2 = (cplx *)xmalloc(sizeof(cplx) * (size_t)p->nv);
        cplx *adj = (cplx *)xmalloc(sizeof(cplx) * (size_t)p->nv);
        for (int64_t k = 0; k < p->n_inst; k++) {
            for (int n = 0; n < p->nv; n++) {
                int op = p->vop[n];
                cplx u = 0, w = 0, v = 0, a1 = 0, a2 = 0;
                if (is_unary(op) || is_binary(op)) u = val[p->va[n]];
                if (is_binary(op)) w = val[p->vb[n]];
                switch (op) {
                case OV_CONST: v = p->vf[n]; break;
                case OV_DATA: v = data_val(p, p->vi[n], k); break;
                case OV_VAR: v = x[idx_eval(p, p->va[n], k)]; break;
                case OV_PARAM: v = m->theta[idx_eval(p, p->va[n], k)]; break;
                case OV_NEG: v = -u; a1 = -1; break;
                case OV_ABS2: v = u * u; a1 = 2.0 * u; break;
                case OV_INV: v = 1.0 / u; a1 = -1.0 / (u * u); break;
                case OV_EXP: v = cexp(u); a1 = v; break;
                case OV_LOG: v = clog(u); a1 = 1.0 / u; break;
                case OV_SIN: v = csin(u); a1 = ccos(u); break;
                case OV_COS: v = ccos(u); a1 = -csin(u); break;
                case OV_SQRT: v = csqrt(u); a1 = 0.5 / v; break;
                case OV_TAN: { cplx c = ccos(u); v = ctan(u); a1 = 1.0 / (c * c); break; }
                case OV_TANH: v = ctanh(u); a1 = 1.0 - v * v; break;
                case OV_ATAN: v = catan(u); a1 = 1.0 / (1.0 + u * u); break;
                case OV_POWI: v = cipow(u, p->vi[n]); a1 = (double)p->vi[n] * cipow(u, p->vi[n] - 1); break;
                case OV_SINH: v = csinh(u); a1 = ccosh(u); break;
                case OV_COSH: v = ccosh(u); a1 = csinh(u); break;
                case OV_ASIN: v = casin(u); a1 = 1.0 / csqrt(1.0 - u * u); break;
                case OV_ACOS: v = cacos(u); a1 = -1.0 / csqrt(1.0 - u * u); break;
                case OV_LOG1P: v = clog(1.0 + u); a1 = 1.0 / (1.0 + u); break;
                case OV_EXPM1: v = cexp(u) - 1.0; a1 = cexp(u); break;
                case OV_LOG2: v = clog(u) / log(2.0); a1 = 1.0 / (u * log(2.0)); break;
                case OV_LOG10: v = clog(u) / log(10.0); a1 = 1.0 / (u * log(10.0)); break;
                case OV_EXP2: v = cexp(u * log(2.0)); a1 = v * log(2.0); break;
                case OV_ATAN2: v = catan2_(u, w); a1 = w / (u * u + w * w); a2 = -u / (u * u + w * w); break;
                case OV_HYPOT: v = csqrt(u * u + w * w); a1 = u / v; a2 = w / v; break;
                case OV_ADD: v = u + w; a1 = 1; a2 = 1; break;
                case OV_SUB: v = u - w; a1 = 1; a2 = -1; break;
                case OV_MUL: v = u * w; a1 = w; a2 = u; break;
                case OV_DIV: v = u / w; a1 = 1.0 / w; a2 = -u / (w * w); break;
                case OV_POW: v = cexp(w * clog(u)); a1 = w * cexp((w - 1.0) * clog(u)); a2 = v * clog(u); break;
                }
                val[n] = v; d1[n] = a1; d2[n] = a2; adj[n] = 0;
            }
            double wgt = p->kind == OK_OBJ ? sigma : y[pattern_row(p, k)];
            adj[p->nv - 1] = wgt;
            for (int n = p->nv - 1; n >= 0; n--) {
                int op = p->vop[n];
                if (op == OV_VAR) g[idx_eval(p, p->va[n], k)] += adj[n];
                else if (is_unary(op)) adj[p->va[n]] += adj[n] * d1[n];
                else if (is_binary(op)) { adj[p->va[n]] += adj[n] * d1[n]; adj[p->vb[n]] += adj[n] * d2[n]; }
            }
        }
        free(val); free(d1); free(d2); free(adj);
    }
    for (int64_t v = 0; v < m->nvar; v++) { gr[v] = creal(g[v]); gi[v] = cimag(g[v]); }
    free(x); free(g);
    return ORC_OK;
}

/* ------------------------------------------------------------------ teardown */
void orc_free(orc_model *m) {
    if (!m) return;
    for (int i = 0; i < m->np; i++) {
        opat *p = &m->p[i];
        void *arrs[] = {p->vop, p->va, p->vb, p->vi, p->vf, p->iop, p->ia, p->ib, p->ii, p->ftype,
                        (void *)p->fptr, p->sym_of, p->sym_root, p->raw1, p->comp1, p->jsym,
                        p->raw2a, p->raw2b, p->comp2, p->ha, p->hb};
        for (size_t j = 0; j < sizeof arrs / sizeof arrs[0]; j++) free(arrs[j]);
    }
    free(m->p); free(m->theta);
    void *arrs[] = {m->jrow, m->jcol, m->hrow, m->hcol, m->j_colptr, m->j_rowval, m->j_coo2csc,
                    m->h_colptr, m->h_rowval, m->h_coo2csc};
    for (size_t j = 0; j < sizeof arrs / sizeof arrs[0]; j++) free(arrs[j]);
    free(m);
}
