// exa_lower.cpp -- host-side lowering of the pattern IR to generated CUDA code.
//
//  1. analyse_pattern: validates one pattern tree and computes its symbols and slot tables.
//     Symbols are Var leaves with identical index subtrees (Sec. 4.2.2).  First-order slots are the
//     symbols in the order a reverse pass meets their leaves (pre-order, left operand first;
//     Sec. 5.2.1).  Hessian slots follow the reverse-over-reverse pass of Sec. 5.1.3 structurally:
//     a child's second adjoint is possibly nonzero if its parent's is or the parent's own second
//     partial for that child is not identically zero; leaves with a possibly nonzero second
//     adjoint give a diagonal entry; a binary node, once both children are done, gives every
//     (leaf of child 1) x (leaf of child 2) pair if its own second adjoint or mixed second partial
//     is possibly nonzero.  Entries are deduplicated as unordered symbol pairs (the Compressor of
//     Sec. 5.2.2).
//
//  2. generate_source: builds, per pattern, a hash-consed expression graph holding the value, the
//     reverse-mode first derivatives and the second derivatives obtained by reverse over reverse
//     (edge pushing: second adjoints pushed to the leaves, cross terms at binary nodes weighted by
//     products of subtree gradients), with structurally zero terms removed at construction
//     (Sec. 7.2.2, affine-node specialisation).  It then prints straight-line CUDA code per
//     (pattern, callback), one kernel per callback over a tile list, for NVRTC.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <iterator>
#include <map>
#include <set>
#include <sstream>
#include <tuple>

#include "exa_internal.h"

namespace exa {

#define EXA_STR2(...) #__VA_ARGS__
#define EXA_STR(...) EXA_STR2(__VA_ARGS__)
const char *const kDeviceStructs = EXA_STR(EXA_DEVICE_STRUCTS);
const char *const kModeName[M_COUNT] = {"obj", "con", "grad", "jac", "hess", "all", "first", "struct",
                                        "hess_c", "hess_b", "all_c", "all_b"};

static bool is_unary(int op) { return op >= EXA_V_NEG && op <= EXA_V_EXP2; }
static bool is_binary(int op) { return op >= EXA_V_ADD && op <= EXA_V_HYPOT; }
static bool is_leaf(int op) { return op >= EXA_V_CONST && op <= EXA_V_PARAM; }

// Is the op's second partial identically zero?  which: 1 = d2/du1^2, 2 = d2/du2^2, 3 = mixed.
static bool second_partial_nonzero(const VNode &n, int which) {
    switch (n.op) {
    case EXA_V_NEG: case EXA_V_ADD: case EXA_V_SUB: return false;
    case EXA_V_POWI: return !(n.iv == 0 || n.iv == 1);
    case EXA_V_MUL: return which == 3;
    case EXA_V_DIV: return which != 1;
    default: return true;
    }
}

// ------------------------------------------------------------------ index-expression keys
static std::string idx_key(const std::vector<INode> &ix, int r) {
    const INode &n = ix[r];
    switch (n.op) {
    case EXA_I_CONST: return "c" + std::to_string(n.iv);
    case EXA_I_FIELD: return "f" + std::to_string(n.iv);
    case EXA_I_INST: return "k";
    default: {
        const char *o = n.op == EXA_I_ADD ? "+" : n.op == EXA_I_SUB ? "-" : "*";
        return std::string("(") + idx_key(ix, n.a) + o + idx_key(ix, n.b) + ")";
    }
    }
}

std::vector<int> symbol_partition(const Pattern &p, const std::vector<INode> &ix) {
    const int nv = (int)p.v.size();
    std::vector<int> out(nv, -1);
    std::map<std::string, int> ids;
    std::vector<int> stack{nv - 1};
    while (!stack.empty()) {
        int i = stack.back();
        stack.pop_back();
        const VNode &n = p.v[i];
        if (n.op == EXA_V_VAR) {
            auto r = ids.emplace(idx_key(ix, n.a), (int)ids.size());
            out[i] = r.first->second;
        } else if (is_unary(n.op)) {
            stack.push_back(n.a);
        } else if (is_binary(n.op)) {
            stack.push_back(n.b);
            stack.push_back(n.a);
        }
    }
    return out;
}

static std::string check_idx(const Pattern &p, int r, int limit, int depth = 0) {
    if (depth > 64) return "index expression too deep";
    if (r < 0 || r >= limit) return "index node reference out of range or not before its parent";
    const INode &n = p.ix[r];
    switch (n.op) {
    case EXA_I_CONST: case EXA_I_INST: return "";
    case EXA_I_FIELD:
        if (n.iv < 0 || n.iv >= (long long)p.ftype.size() || p.ftype[n.iv] != EXA_FIELD_I32)
            return "index expression reads a missing or non-int32 data field";
        return "";
    case EXA_I_ADD: case EXA_I_SUB: case EXA_I_MUL: {
        std::string e = check_idx(p, n.a, r, depth + 1);
        return e.empty() ? check_idx(p, n.b, r, depth + 1) : e;
    }
    default: return "unknown index opcode";
    }
}

std::string analyse_pattern(Pattern &p) {
    const int nv = (int)p.v.size();
    if (p.kind < EXA_OBJ || p.kind > EXA_AUG) return "bad pattern kind";
    if (p.n_inst < 0) return "negative instance count";
    if (p.n_inst >= (1LL << 31)) return "more than 2^31-1 instances in one pattern";
    if (nv < 1) return "empty pattern tree";
    if ((int)p.ftype.size() > EXA_MAXF) return "more than 16 data fields in one pattern";
    for (int t : p.ftype)
        if (t != EXA_FIELD_I32 && t != EXA_FIELD_F64) return "bad data field type";
    // opcodes, child order, tree shape (every non-root node has exactly one parent)
    std::vector<int> parents(nv, 0);
    for (int i = 0; i < nv; i++) {
        const VNode &n = p.v[i];
        if (n.op == EXA_V_CONST) continue;
        if (n.op == EXA_V_DATA) {
            if (n.iv < 0 || n.iv >= (long long)p.ftype.size()) return "data field out of range";
            continue;
        }
        if (n.op == EXA_V_VAR || n.op == EXA_V_PARAM) {
            std::string e = check_idx(p, n.a, (int)p.ix.size());
            if (!e.empty()) return e;
            continue;
        }
        if (is_unary(n.op)) {
            if (n.a < 0 || n.a >= i) return "child must precede its parent";
            parents[n.a]++;
            if (n.op == EXA_V_POWI && (n.iv > 64 || n.iv < -64)) return "integer power beyond +-64";
            continue;
        }
        if (is_binary(n.op)) {
            if (n.a < 0 || n.a >= i || n.b < 0 || n.b >= i) return "child must precede its parent";
            parents[n.a]++;
            parents[n.b]++;
            continue;
        }
        return "unknown value opcode";
    }
    for (int i = 0; i < nv - 1; i++)
        if (parents[i] != 1) return "value nodes must form a tree rooted at the last node";
    if (parents[nv - 1] != 0) return "the root must not have a parent";
    if (p.kind == EXA_AUG) {
        std::string e = check_idx(p, p.row_root, (int)p.ix.size());
        if (!e.empty()) return "augmentation row: " + e;
        if (p.row_limit <= 0 && p.n_inst > 0) return "augmentation target block is empty";
    }

    // symbols by first occurrence in pre-order (left operand first)
    p.sym_of.assign(nv, -1);
    p.sym_root.clear();
    std::map<std::string, int> sym_by_key;
    std::vector<int> preorder_leaves;  // VAR nodes in pre-order
    {
        std::vector<int> stack{nv - 1};
        while (!stack.empty()) {
            int i = stack.back();
            stack.pop_back();
            const VNode &n = p.v[i];
            if (n.op == EXA_V_VAR) {
                preorder_leaves.push_back(i);
            } else if (is_unary(n.op)) {
                stack.push_back(n.a);
            } else if (is_binary(n.op)) {
                stack.push_back(n.b);
                stack.push_back(n.a);
            }
        }
    }
    for (int i : preorder_leaves) {
        std::string key = idx_key(p.ix, p.v[i].a);
        auto it = sym_by_key.find(key);
        int s;
        if (it == sym_by_key.end()) {
            s = (int)p.sym_root.size();
            sym_by_key[key] = s;
            p.sym_root.push_back(p.v[i].a);
        } else {
            s = it->second;
        }
        p.sym_of[i] = s;
    }
    p.nsym = (int)p.sym_root.size();
    // first-order slots: unique symbols in visit order == symbol ids in order
    p.jsym.resize(p.nsym);
    for (int s = 0; s < p.nsym; s++) p.jsym[s] = s;

    // Hessian slots
    std::vector<char> has_var(nv, 0);
    std::vector<std::vector<int>> leaves(nv);  // symbols of Var leaves in pre-order
    for (int i = 0; i < nv; i++) {
        const VNode &n = p.v[i];
        if (n.op == EXA_V_VAR) {
            has_var[i] = 1;
            leaves[i] = {p.sym_of[i]};
        } else if (is_unary(n.op)) {
            has_var[i] = has_var[n.a];
            leaves[i] = leaves[n.a];
        } else if (is_binary(n.op)) {
            has_var[i] = has_var[n.a] || has_var[n.b];
            leaves[i] = leaves[n.a];
            leaves[i].insert(leaves[i].end(), leaves[n.b].begin(), leaves[n.b].end());
        }
    }
    std::vector<char> z2(nv, 0);  // "second adjoint possibly nonzero", set top-down
    for (int i = nv - 1; i >= 0; i--) {
        const VNode &n = p.v[i];
        if (is_unary(n.op)) z2[n.a] = z2[i] || second_partial_nonzero(n, 1);
        else if (is_binary(n.op)) {
            z2[n.a] = z2[i] || second_partial_nonzero(n, 1);
            z2[n.b] = z2[i] || second_partial_nonzero(n, 2);
        }
    }
    p.hpair.clear();
    std::set<std::pair<int, int>> seen;
    auto emit = [&](int a, int b) {
        std::pair<int, int> key(std::min(a, b), std::max(a, b));
        if (seen.insert(key).second) p.hpair.emplace_back(a, b);
    };
    // post-order traversal from the root: children (left, right), then the node itself
    {
        std::vector<std::pair<int, int>> stack{{nv - 1, 0}};
        while (!stack.empty()) {
            auto &top = stack.back();
            int i = top.first;
            const VNode &n = p.v[i];
            if (top.second == 0) {
                top.second = 1;
                if (is_unary(n.op)) { stack.push_back({n.a, 0}); continue; }
                if (is_binary(n.op)) {
                    int a = n.a, b = n.b;
                    stack.push_back({b, 0});
                    stack.push_back({a, 0});
                    continue;
                }
            }
            stack.pop_back();
            if (n.op == EXA_V_VAR) {
                if (z2[i]) emit(p.sym_of[i], p.sym_of[i]);
            } else if (is_binary(n.op) && has_var[n.a] && has_var[n.b] &&
                       (z2[i] || second_partial_nonzero(n, 3))) {
                for (int a : leaves[n.a])
                    for (int b : leaves[n.b]) emit(a, b);
            }
        }
    }
    return "";
}

// ------------------------------------------------------------------ expression graph
namespace {

enum SOp {
    S_LIT, S_IN, S_NEG, S_ADD, S_SUB, S_MUL, S_DIV,
    S_EXP, S_LOG, S_SIN, S_COS, S_SQRT, S_TAN, S_TANH, S_ATAN, S_POW,
    S_CVT,              // convert the operand to this node's precision
    S_SINR, S_COSR,     // float sin / cos of an FP64 argument reduced in FP64
    S_EXPR,             // float exp of an FP64 argument reduced in FP64
    S_SINH, S_COSH, S_ASIN, S_ACOS, S_LOG1P, S_EXPM1, S_LOG2, S_LOG10, S_EXP2,  // unary functions
    S_ATAN2, S_HYPOT    // binary functions
};
enum Prec { PD = 0, PF = 1 };  // FP64, FP32

struct SN {
    int op;
    int prec;
    int a, b;
    double lit;
    char ikind;  // S_IN: 'X' variable symbol, 'D' data field, 'P' parameter node, 'C' member constant
    int iid;
};

class Graph {
  public:
    typedef std::tuple<int, int, int, uint64_t> Key;
    std::vector<SN> n;
    std::map<Key, int> memo;
    std::vector<Key> keys;  // memo key of every node, for rollback
    // Product view of MUL nodes: (precision, sorted factor multiset) -> (node, sign), node = sign x
    // the product of the factors (factors: the non-MUL, non-NEG leaves of the node's product tree).
    std::map<std::pair<int, std::vector<int>>, std::pair<int, int>> prods;
    std::vector<std::pair<int, std::vector<int>>> prod_key;  // per node: the prods entry it registered
    bool factoring = true;

    int make(const SN &s, const Key &key) {
        n.push_back(s);
        keys.push_back(key);
        prod_key.emplace_back(-1, std::vector<int>());
        const int id = (int)n.size() - 1;
        memo[key] = id;
        if (s.op == S_MUL) {
            int sg = 1;
            std::vector<int> f;
            flat(id, sg, f);
            std::sort(f.begin(), f.end());
            auto pk = std::make_pair(s.prec, f);
            if (!prods.count(pk)) {
                prods[pk] = {id, sg};
                prod_key[id] = pk;
            }
        }
        return id;
    }
    // Drops every node created after `mark` (a tentative rewrite that did not pay off).
    void rollback(size_t mark) {
        for (size_t i = n.size(); i-- > mark;) {
            memo.erase(keys[i]);
            if (prod_key[i].first >= 0) prods.erase(prod_key[i]);
        }
        n.resize(mark);
        keys.resize(mark);
        prod_key.resize(mark);
    }
    void flat(int i, int &sg, std::vector<int> &f) const {
        const SN &s = n[i];
        if (s.op == S_NEG) { sg = -sg; flat(s.a, sg, f); }
        else if (s.op == S_MUL) { flat(s.a, sg, f); flat(s.b, sg, f); }
        else f.push_back(i);
    }
    bool find_prod(int prec, const std::vector<int> &f, int &node, int &sign) const {
        if (f.size() == 1) { node = f[0]; sign = 1; return true; }
        auto it = prods.find(std::make_pair(prec, f));
        if (it == prods.end()) return false;
        node = it->second.first;
        sign = it->second.second;
        return true;
    }
    // Distributive rewrite of a +- b when both are products with common factors C:
    // C * (rest_a +- rest_b), tried only when C, rest_a and rest_b already exist as nodes, and kept
    // only when it needs at most one new arithmetic node (the plain sum needs one): typically the
    // rewritten form is an existing node, e.g. the second adjoints that sin and cos of one argument
    // push to it, x1 x2 (b sin t) + x1 x2 (g cos t), are x1 x2 (g cos t + b sin t), which the primal
    // value already computed.  Exact in real arithmetic; only the rounding differs.
    int try_factor(int a, int b, bool subtract) {
        if (!factoring || n[a].prec != n[b].prec) return -1;
        const int prec = n[a].prec;
        int sa = 1, sb = subtract ? -1 : 1;
        std::vector<int> fa, fb, common, ra, rb;
        flat(a, sa, fa);
        flat(b, sb, fb);
        if (fa.size() < 2 || fb.size() < 2) return -1;
        std::sort(fa.begin(), fa.end());
        std::sort(fb.begin(), fb.end());
        std::set_intersection(fa.begin(), fa.end(), fb.begin(), fb.end(), std::back_inserter(common));
        if (common.empty() || common.size() == fa.size() || common.size() == fb.size()) return -1;
        std::set_difference(fa.begin(), fa.end(), common.begin(), common.end(), std::back_inserter(ra));
        std::set_difference(fb.begin(), fb.end(), common.begin(), common.end(), std::back_inserter(rb));
        int pc, sc, pa, sA, pb, sB;
        if (!find_prod(prec, common, pc, sc) || !find_prod(prec, ra, pa, sA) || !find_prod(prec, rb, pb, sB)) return -1;
        const size_t mark = n.size();
        const bool pos_a = sa * sA > 0, pos_b = sb * sB > 0;
        int inner;
        if (pos_a && pos_b) inner = add(pa, pb);
        else if (pos_a) inner = sub(pa, pb);
        else if (pos_b) inner = sub(pb, pa);
        else inner = neg(add(pa, pb));
        int r = mul(pc, inner);
        if (sc < 0) r = neg(r);
        int cost = 0;
        for (size_t i = mark; i < n.size(); i++) cost += n[i].op != S_NEG;
        if (cost > 1) {
            rollback(mark);
            return -1;
        }
        return r;
    }

    int lit(double v, int prec) {
        if (prec == PF) v = (double)(float)v;
        uint64_t bits;
        std::memcpy(&bits, &v, 8);
        auto key = std::make_tuple((int)S_LIT * 2 + prec, -1, -1, bits);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        return make({S_LIT, prec, -1, -1, v, 0, 0}, key);
    }
    int input(char kind, int id, int prec) {
        auto key = std::make_tuple((int)S_IN * 2 + prec, (int)kind, id, (uint64_t)0);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        return make({S_IN, prec, -1, -1, 0.0, kind, id}, key);
    }
    bool has(int op, int prec, int a, int b = -1) const {
        return memo.count(std::make_tuple(op * 2 + prec, a, b, (uint64_t)0)) > 0;
    }
    int node(int op, int prec, int a, int b = -1) {
        auto key = std::make_tuple(op * 2 + prec, a, b, (uint64_t)0);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        return make({op, prec, a, b, 0.0, 0, 0}, key);
    }
    int P(int i) const { return n[i].prec; }
    bool is_lit(int i) const { return n[i].op == S_LIT; }
    bool is(int i, double v) const { return n[i].op == S_LIT && n[i].lit == v; }
    bool zero(int i) const { return is(i, 0.0); }
    double fold(double v, int prec) const { return prec == PF ? (double)(float)v : v; }

    int neg(int a) {
        if (is_lit(a)) return lit(-n[a].lit, P(a));
        if (n[a].op == S_NEG) return n[a].a;
        return node(S_NEG, P(a), a);
    }
    // Negations are pulled outward ((-a) b = -(a b), a + (-b) = a - b, ...; exact in IEEE
    // arithmetic) so that expressions differing only in signs share one node.
    bool isneg(int i) const { return n[i].op == S_NEG; }
    int add(int a, int b) {
        if (zero(a)) return b;
        if (zero(b)) return a;
        if (is_lit(a) && is_lit(b)) return lit(fold(n[a].lit + n[b].lit, P(a)), P(a));
        if (isneg(b)) return sub(a, n[b].a);
        if (isneg(a)) return sub(b, n[a].a);
        if (a > b) std::swap(a, b);  // a + b == b + a exactly
        if (!has(S_ADD, P(a), a, b)) {
            int f = try_factor(a, b, false);
            if (f >= 0) return f;
        }
        return node(S_ADD, P(a), a, b);
    }
    int sub(int a, int b) {
        if (zero(b)) return a;
        if (zero(a)) return neg(b);
        if (is_lit(a) && is_lit(b)) return lit(fold(n[a].lit - n[b].lit, P(a)), P(a));
        if (isneg(b)) return add(a, n[b].a);
        if (isneg(a)) return neg(add(n[a].a, b));
        if (!has(S_SUB, P(a), std::min(a, b), std::max(a, b))) {
            int f = try_factor(a, b, true);
            if (f >= 0) return f;
        }
        if (a > b) return neg(node(S_SUB, P(a), b, a));  // a - b == -(b - a) exactly: one canonical form
        return node(S_SUB, P(a), a, b);
    }
    int mul(int a, int b) {
        if (zero(a) || zero(b)) return lit(0.0, P(a));
        if (is(a, 1.0)) return b;
        if (is(b, 1.0)) return a;
        if (is(a, -1.0)) return neg(b);
        if (is(b, -1.0)) return neg(a);
        if (is_lit(a) && is_lit(b)) return lit(fold(n[a].lit * n[b].lit, P(a)), P(a));
        if (isneg(a)) return neg(mul(n[a].a, b));
        if (isneg(b)) return neg(mul(a, n[b].a));
        if (a > b) std::swap(a, b);
        return node(S_MUL, P(a), a, b);
    }
    int div(int a, int b) {
        if (is(b, 1.0)) return a;
        if (zero(a)) return lit(0.0, P(a));
        if (is_lit(a) && is_lit(b)) return lit(fold(n[a].lit / n[b].lit, P(a)), P(a));
        if (isneg(a)) return neg(div(n[a].a, b));
        if (isneg(b)) return neg(div(a, n[b].a));
        return node(S_DIV, P(a), a, b);
    }
    int fn(int op, int a) { return fn_at(op, P(a), a); }
    int fn_at(int op, int prec, int a) {
        // sin(-u) = -sin(u), cos(-u) = cos(u): lets sin/cos of opposite arguments share one call
        if (n[a].op == S_NEG && (op == S_SIN || op == S_SINR)) return neg(node(op, prec, n[a].a));
        if (n[a].op == S_NEG && (op == S_COS || op == S_COSR)) return node(op, prec, n[a].a);
        return node(op, prec, a);
    }
    int powi(int u, long long m) {
        if (m == 0) return lit(1.0, P(u));
        if (m < 0) return div(lit(1.0, P(u)), powi(u, -m));
        if (m == 1) return u;
        int h = powi(u, m / 2);
        int sq = mul(h, h);
        return (m % 2) ? mul(sq, u) : sq;
    }
};

struct PatternGraph {
    std::vector<int> val, d1, d2, h11, h12, h22, adj, adj2;
    int value = -1;
    std::vector<int> grad;                    // per pattern symbol
    std::map<std::pair<int, int>, int> hess;  // unordered pattern-symbol pair -> entry
    std::string err;
};

static std::string fmt_double(double v) {
    if (!std::isfinite(v)) {
        uint64_t bits;
        std::memcpy(&bits, &v, 8);
        return "__longlong_as_double(" + std::to_string((long long)bits) + "LL)";
    }
    char buf[64];
    std::snprintf(buf, sizeof buf, "%.17g", v);
    std::string s(buf);
    if (s.find_first_of(".eE") == std::string::npos) s += ".0";
    if (v < 0 || (v == 0 && std::signbit(v))) s = "(" + s + ")";
    return s;
}

static std::string fmt_float(double v) {
    float f = (float)v;
    if (!std::isfinite(f)) {
        uint32_t bits;
        std::memcpy(&bits, &f, 4);
        return "__int_as_float(" + std::to_string((int)bits) + ")";
    }
    char buf[64];
    std::snprintf(buf, sizeof buf, "%.9g", (double)f);
    std::string s(buf);
    if (s.find_first_of(".eE") == std::string::npos) s += ".0";
    s += "f";
    if (f < 0 || (f == 0 && std::signbit(f))) s = "(" + s + ")";
    return s;
}

// Group-level input ids of one pattern: 'X' group symbol, 'D' group column, 'C' constant slot,
// 'P' parameter node (position * 65536 + node).
struct InputMap {
    const std::vector<int> *sym;
    const std::vector<int> *field;
    int pos;
};

// Builds value, gradient over symbols and Hessian over symbol pairs of one pattern into the
// group's shared graph.  FP64 mode: every node in FP64.  Mixed mode: every node in FP32 except the
// primal subtrees that form the arguments of sin / cos / tan / exp, evaluated and reduced in FP64.
static void build_graph(const Pattern &p, const InputMap &im, Graph &g, PatternGraph &G, bool mixed) {
    const int nv = (int)p.v.size();
    const int W = mixed ? PF : PD;  // working precision of pattern arithmetic
    G.val.assign(nv, -1);
    int Z = g.lit(0.0, W), ONE = g.lit(1.0, W), TWO = g.lit(2.0, W);
    G.d1.assign(nv, Z); G.d2.assign(nv, Z);
    G.h11.assign(nv, Z); G.h12.assign(nv, Z); G.h22.assign(nv, Z);
    std::vector<char> hv(nv, 0);
    auto X = [&](int i, int prec) { return g.input('X', (*im.sym)[p.sym_of[i]], prec); };
    auto D = [&](int f, int prec) { return g.input('D', (*im.field)[f], prec); };
    auto Pm = [&](int i, int prec) { return g.input('P', im.pos * 65536 + i, prec); };
    auto K = [&](int i, int prec) {
        auto it = p.fvary.find(i);
        return it != p.fvary.end() ? g.input('C', it->second, prec) : g.lit(p.v[i].fv, prec);
    };
    // FP64 primal value of a subtree (argument formation in mixed mode)
    std::vector<int> dmemo(nv, -1);
    std::function<int(int)> dval = [&](int i) -> int {
        if (dmemo[i] >= 0) return dmemo[i];
        const VNode &nd = p.v[i];
        int r = -1;
        switch (nd.op) {
        case EXA_V_CONST: r = K(i, PD); break;
        case EXA_V_DATA: r = D((int)nd.iv, PD); break;
        case EXA_V_VAR: r = X(i, PD); break;
        case EXA_V_PARAM: r = Pm(i, PD); break;
        case EXA_V_NEG: r = g.neg(dval(nd.a)); break;
        case EXA_V_ABS2: { int u = dval(nd.a); r = g.mul(u, u); break; }
        case EXA_V_INV: r = g.div(g.lit(1.0, PD), dval(nd.a)); break;
        case EXA_V_EXP: r = g.fn(S_EXP, dval(nd.a)); break;
        case EXA_V_LOG: r = g.fn(S_LOG, dval(nd.a)); break;
        case EXA_V_SIN: r = g.fn(S_SIN, dval(nd.a)); break;
        case EXA_V_COS: r = g.fn(S_COS, dval(nd.a)); break;
        case EXA_V_SQRT: r = g.fn(S_SQRT, dval(nd.a)); break;
        case EXA_V_TAN: r = g.fn(S_TAN, dval(nd.a)); break;
        case EXA_V_TANH: r = g.fn(S_TANH, dval(nd.a)); break;
        case EXA_V_ATAN: r = g.fn(S_ATAN, dval(nd.a)); break;
        case EXA_V_POWI: r = g.powi(dval(nd.a), nd.iv); break;
        case EXA_V_ADD: r = g.add(dval(nd.a), dval(nd.b)); break;
        case EXA_V_SUB: r = g.sub(dval(nd.a), dval(nd.b)); break;
        case EXA_V_MUL: r = g.mul(dval(nd.a), dval(nd.b)); break;
        case EXA_V_DIV: r = g.div(dval(nd.a), dval(nd.b)); break;
        case EXA_V_POW: r = g.node(S_POW, PD, dval(nd.a), dval(nd.b)); break;
        case EXA_V_SINH: r = g.fn(S_SINH, dval(nd.a)); break;
        case EXA_V_COSH: r = g.fn(S_COSH, dval(nd.a)); break;
        case EXA_V_ASIN: r = g.fn(S_ASIN, dval(nd.a)); break;
        case EXA_V_ACOS: r = g.fn(S_ACOS, dval(nd.a)); break;
        case EXA_V_LOG1P: r = g.fn(S_LOG1P, dval(nd.a)); break;
        case EXA_V_EXPM1: r = g.fn(S_EXPM1, dval(nd.a)); break;
        case EXA_V_LOG2: r = g.fn(S_LOG2, dval(nd.a)); break;
        case EXA_V_LOG10: r = g.fn(S_LOG10, dval(nd.a)); break;
        case EXA_V_EXP2: r = g.fn(S_EXP2, dval(nd.a)); break;
        case EXA_V_ATAN2: r = g.node(S_ATAN2, PD, dval(nd.a), dval(nd.b)); break;
        case EXA_V_HYPOT: r = g.node(S_HYPOT, PD, dval(nd.a), dval(nd.b)); break;
        }
        return dmemo[i] = r;
    };
    for (int i = 0; i < nv; i++) {
        const VNode &nd = p.v[i];
        int u = nd.a >= 0 && !is_leaf(nd.op) ? G.val[nd.a] : -1;
        int w = nd.b >= 0 && is_binary(nd.op) ? G.val[nd.b] : -1;
        int v = Z, d1 = Z, d2 = Z, h11 = Z, h12 = Z, h22 = Z;
        switch (nd.op) {
        case EXA_V_CONST: v = K(i, W); break;
        case EXA_V_DATA: v = D((int)nd.iv, W); break;
        case EXA_V_VAR: v = X(i, W); hv[i] = 1; break;
        case EXA_V_PARAM: v = Pm(i, W); break;
        case EXA_V_NEG: v = g.neg(u); d1 = g.lit(-1.0, W); break;
        case EXA_V_ABS2: v = g.mul(u, u); d1 = g.mul(TWO, u); h11 = TWO; break;
        case EXA_V_INV:
            v = g.div(ONE, u);
            d1 = g.neg(g.mul(v, v));
            h11 = g.mul(TWO, g.mul(v, g.mul(v, v)));
            break;
        case EXA_V_EXP:
            v = mixed ? g.fn_at(S_EXPR, PF, dval(nd.a)) : g.fn(S_EXP, u);
            d1 = v; h11 = v;
            break;
        case EXA_V_LOG: v = g.fn(S_LOG, u); d1 = g.div(ONE, u); h11 = g.neg(g.mul(d1, d1)); break;
        case EXA_V_SIN:
            if (mixed) { v = g.fn_at(S_SINR, PF, dval(nd.a)); d1 = g.fn_at(S_COSR, PF, dval(nd.a)); }
            else { v = g.fn(S_SIN, u); d1 = g.fn(S_COS, u); }
            h11 = g.neg(v);
            break;
        case EXA_V_COS:
            if (mixed) { v = g.fn_at(S_COSR, PF, dval(nd.a)); d1 = g.neg(g.fn_at(S_SINR, PF, dval(nd.a))); }
            else { v = g.fn(S_COS, u); d1 = g.neg(g.fn(S_SIN, u)); }
            h11 = g.neg(v);
            break;
        case EXA_V_SQRT:
            v = g.fn(S_SQRT, u);
            d1 = g.div(g.lit(0.5, W), v);
            h11 = g.neg(g.div(g.lit(0.25, W), g.mul(u, v)));
            break;
        case EXA_V_TAN:
            v = mixed ? g.div(g.fn_at(S_SINR, PF, dval(nd.a)), g.fn_at(S_COSR, PF, dval(nd.a))) : g.fn(S_TAN, u);
            d1 = g.add(ONE, g.mul(v, v));
            h11 = g.mul(TWO, g.mul(v, d1));
            break;
        case EXA_V_TANH: v = g.fn(S_TANH, u); d1 = g.sub(ONE, g.mul(v, v)); h11 = g.mul(g.lit(-2.0, W), g.mul(v, d1)); break;
        case EXA_V_ATAN:
            v = g.fn(S_ATAN, u);
            d1 = g.div(ONE, g.add(ONE, g.mul(u, u)));
            h11 = g.mul(g.lit(-2.0, W), g.mul(u, g.mul(d1, d1)));
            break;
        case EXA_V_POWI:
            v = g.powi(u, nd.iv);
            d1 = g.mul(g.lit((double)nd.iv, W), g.powi(u, nd.iv - 1));
            h11 = g.mul(g.lit((double)nd.iv * (double)(nd.iv - 1), W), g.powi(u, nd.iv - 2));
            break;
        // exp-family functions in mixed mode: value and first derivative evaluated in FP64 from the
        // FP64 argument and rounded to FP32 (the exp arguments are reduced in FP64)
        case EXA_V_SINH: case EXA_V_COSH: {
            const int o1 = nd.op == EXA_V_SINH ? S_SINH : S_COSH, o2 = nd.op == EXA_V_SINH ? S_COSH : S_SINH;
            if (mixed) { v = g.node(S_CVT, PF, g.fn(o1, dval(nd.a))); d1 = g.node(S_CVT, PF, g.fn(o2, dval(nd.a))); }
            else { v = g.fn(o1, u); d1 = g.fn(o2, u); }
            h11 = v;
            break;
        }
        case EXA_V_EXPM1:
            if (mixed) { v = g.node(S_CVT, PF, g.fn(S_EXPM1, dval(nd.a))); d1 = g.fn_at(S_EXPR, PF, dval(nd.a)); }
            else { v = g.fn(S_EXPM1, u); d1 = g.fn(S_EXP, u); }
            h11 = d1;
            break;
        case EXA_V_EXP2: {
            const int ln2 = g.lit(0.69314718055994531, W);
            v = mixed ? g.node(S_CVT, PF, g.fn(S_EXP2, dval(nd.a))) : g.fn(S_EXP2, u);
            d1 = g.mul(v, ln2);
            h11 = g.mul(d1, ln2);
            break;
        }
        case EXA_V_ASIN: case EXA_V_ACOS: {
            const int r = g.div(ONE, g.fn(S_SQRT, g.sub(ONE, g.mul(u, u))));
            v = g.fn(nd.op == EXA_V_ASIN ? S_ASIN : S_ACOS, u);
            d1 = nd.op == EXA_V_ASIN ? r : g.neg(r);
            h11 = g.mul(u, g.mul(d1, g.mul(r, r)));
            break;
        }
        case EXA_V_LOG1P: v = g.fn(S_LOG1P, u); d1 = g.div(ONE, g.add(ONE, u)); h11 = g.neg(g.mul(d1, d1)); break;
        case EXA_V_LOG2: case EXA_V_LOG10: {
            const int lnb = g.lit(nd.op == EXA_V_LOG2 ? 0.69314718055994531 : 2.3025850929940457, W);
            v = g.fn(nd.op == EXA_V_LOG2 ? S_LOG2 : S_LOG10, u);
            d1 = g.div(ONE, g.mul(u, lnb));
            h11 = g.neg(g.div(d1, u));
            break;
        }
        case EXA_V_ATAN2: {
            v = g.node(S_ATAN2, W, u, w);
            const int r = g.add(g.mul(u, u), g.mul(w, w));
            const int r2 = g.mul(r, r);
            d1 = g.div(w, r);
            d2 = g.neg(g.div(u, r));
            h11 = g.neg(g.div(g.mul(TWO, g.mul(u, w)), r2));
            h12 = g.div(g.sub(g.mul(u, u), g.mul(w, w)), r2);
            h22 = g.div(g.mul(TWO, g.mul(u, w)), r2);
            break;
        }
        case EXA_V_HYPOT: {
            v = g.node(S_HYPOT, W, u, w);
            const int v3 = g.mul(v, g.mul(v, v));
            d1 = g.div(u, v);
            d2 = g.div(w, v);
            h11 = g.div(g.mul(w, w), v3);
            h12 = g.neg(g.div(g.mul(u, w), v3));
            h22 = g.div(g.mul(u, u), v3);
            break;
        }
        case EXA_V_ADD: v = g.add(u, w); d1 = ONE; d2 = ONE; break;
        case EXA_V_SUB: v = g.sub(u, w); d1 = ONE; d2 = g.lit(-1.0, W); break;
        case EXA_V_MUL: v = g.mul(u, w); d1 = w; d2 = u; h12 = ONE; break;
        case EXA_V_DIV: {
            v = g.div(u, w);
            int r = g.div(ONE, w);
            d1 = r;
            d2 = g.neg(g.mul(v, r));
            h12 = g.neg(g.mul(r, r));
            h22 = g.mul(TWO, g.mul(v, g.mul(r, r)));
            break;
        }
        case EXA_V_POW: {
            v = g.node(S_POW, W, u, w);
            int lu = g.fn(S_LOG, u);
            int vu = g.div(v, u);
            d1 = g.mul(w, vu);
            d2 = g.mul(v, lu);
            h11 = g.mul(g.mul(w, g.sub(w, ONE)), g.div(vu, u));
            h12 = g.mul(vu, g.add(ONE, g.mul(w, lu)));
            h22 = g.mul(v, g.mul(lu, lu));
            break;
        }
        }
        if (is_unary(nd.op)) hv[i] = hv[nd.a];
        if (is_binary(nd.op)) hv[i] = hv[nd.a] || hv[nd.b];
        G.val[i] = v; G.d1[i] = d1; G.d2[i] = d2; G.h11[i] = h11; G.h12[i] = h12; G.h22[i] = h22;
    }
    // Mixed mode: an objective term's value is evaluated in FP64 (dval).  The objective is one sum
    // over all terms, and terms of opposite sign cancel: an FP32 rounding of each term, however
    // exactly the terms are summed afterwards, would leave the sum with far more than FP32's
    // relative error.  Its derivatives are per-variable outputs and stay FP32.
    G.value = (mixed && p.kind == EXA_OBJ) ? dval(nv - 1) : G.val[nv - 1];

    // first-order reverse pass (adjoints), then second order by edge pushing with tangent gradients
    G.adj.assign(nv, Z);
    G.adj2.assign(nv, Z);
    G.grad.assign(p.nsym, Z);
    G.adj[nv - 1] = ONE;
    std::vector<std::map<int, int>> tg(nv);  // subtree gradient over pattern symbols (bottom-up)
    for (int i = 0; i < nv; i++) {
        const VNode &nd = p.v[i];
        if (nd.op == EXA_V_VAR) tg[i][p.sym_of[i]] = ONE;
        else if (is_unary(nd.op)) {
            for (auto &kv : tg[nd.a]) tg[i][kv.first] = g.mul(G.d1[i], kv.second);
        } else if (is_binary(nd.op)) {
            for (auto &kv : tg[nd.a]) tg[i][kv.first] = g.mul(G.d1[i], kv.second);
            for (auto &kv : tg[nd.b]) {
                int t = g.mul(G.d2[i], kv.second);
                auto it = tg[i].find(kv.first);
                if (it == tg[i].end()) tg[i][kv.first] = t;
                else it->second = g.add(it->second, t);
            }
        }
    }
    auto hacc = [&](int s, int t, int c) {
        std::pair<int, int> key(std::min(s, t), std::max(s, t));
        auto it = G.hess.find(key);
        if (it == G.hess.end()) G.hess[key] = c;
        else it->second = g.add(it->second, c);
    };
    for (int i = nv - 1; i >= 0; i--) {
        const VNode &nd = p.v[i];
        int a1 = G.adj[i], a2 = G.adj2[i];
        if (nd.op == EXA_V_VAR) {
            int s = p.sym_of[i];
            G.grad[s] = g.add(G.grad[s], a1);
            if (!g.zero(a2)) hacc(s, s, a2);
        } else if (is_unary(nd.op)) {
            if (!hv[nd.a]) continue;
            G.adj[nd.a] = g.mul(a1, G.d1[i]);
            G.adj2[nd.a] = g.add(g.mul(a2, g.mul(G.d1[i], G.d1[i])), g.mul(a1, G.h11[i]));
        } else if (is_binary(nd.op)) {
            if (hv[nd.a]) {
                G.adj[nd.a] = g.mul(a1, G.d1[i]);
                G.adj2[nd.a] = g.add(g.mul(a2, g.mul(G.d1[i], G.d1[i])), g.mul(a1, G.h11[i]));
            }
            if (hv[nd.b]) {
                G.adj[nd.b] = g.mul(a1, G.d2[i]);
                G.adj2[nd.b] = g.add(g.mul(a2, g.mul(G.d2[i], G.d2[i])), g.mul(a1, G.h22[i]));
            }
            if (hv[nd.a] && hv[nd.b]) {
                int w = g.add(g.mul(a2, g.mul(G.d1[i], G.d2[i])), g.mul(a1, G.h12[i]));
                if (g.zero(w)) continue;
                for (auto &ka : tg[nd.a])
                    for (auto &kb : tg[nd.b]) {
                        int c = g.mul(w, g.mul(ka.second, kb.second));
                        if (ka.first == kb.first) c = g.mul(TWO, c);
                        hacc(ka.first, kb.first, c);
                    }
            }
        }
    }
    std::set<std::pair<int, int>> slots;
    for (auto &pr : p.hpair) slots.insert({std::min(pr.first, pr.second), std::max(pr.first, pr.second)});
    for (auto &kv : G.hess)
        if (!g.zero(kv.second) && !slots.count(kv.first)) {
            G.err = "internal: second-order entry outside the structural slots";
            return;
        }
}

}  // namespace

// ------------------------------------------------------------------ group symbols
static std::string group_idx_key(const Pattern &p, const std::vector<int> &field, int r) {
    const INode &n = p.ix[r];
    switch (n.op) {
    case EXA_I_CONST: {
        auto it = p.ivary.find(r);
        if (it != p.ivary.end()) return "v" + std::to_string(it->second);
        return "c" + std::to_string(n.iv);
    }
    case EXA_I_FIELD: return "f" + std::to_string(field[n.iv]);
    case EXA_I_INST: return "k";
    default: {
        const char *o = n.op == EXA_I_ADD ? "+" : n.op == EXA_I_SUB ? "-" : "*";
        return std::string("(") + group_idx_key(p, field, n.a) + o + group_idx_key(p, field, n.b) + ")";
    }
    }
}

void finalize_group(Group &g, const std::vector<Pattern> &pats) {
    std::map<std::string, int> ids;
    g.sym.assign(g.pats.size(), {});
    g.sym_root.clear();
    for (size_t pos = 0; pos < g.pats.size(); pos++) {
        const Pattern &p = pats[g.pats[pos]];
        g.sym[pos].resize(p.nsym);
        for (int s = 0; s < p.nsym; s++) {
            auto r = ids.emplace(group_idx_key(p, g.field[pos], p.sym_root[s]), (int)ids.size());
            if (r.second) g.sym_root.push_back({(int)pos, p.sym_root[s]});
            g.sym[pos][s] = r.first->second;
        }
    }
    g.hc.clear();
    g.hc_sym.clear();
    std::map<std::pair<int, int>, int> slot;
    for (size_t pos = 0; pos < g.pats.size(); pos++) {
        const Pattern &p = pats[g.pats[pos]];
        for (int j = 0; j < p.nh(); j++) {
            int a = g.sym[pos][p.hpair[j].first], b = g.sym[pos][p.hpair[j].second];
            auto r = slot.emplace(std::make_pair(std::min(a, b), std::max(a, b)), (int)g.hc.size());
            if (r.second) {
                g.hc.emplace_back();
                g.hc_sym.push_back(r.first->first);
            }
            g.hc[r.first->second].push_back({(int)pos, j});
        }
    }
}

bool pattern_in_mode(const Pattern &p, Mode m) {
    switch (m) {
    case M_OBJ: case M_GRAD: return p.kind == EXA_OBJ;
    case M_CON: case M_JAC: return p.kind != EXA_OBJ;
    case M_HESS: case M_HESS_C: case M_HESS_B: return p.nh() > 0;
    default: return true;
    }
}

std::vector<std::vector<int>> group_sets(const std::vector<Pattern> &pats, const Group &g, Mode mode, int lanes) {
    std::vector<int> act;
    for (size_t pos = 0; pos < g.pats.size(); pos++)
        if (pattern_in_mode(pats[g.pats[pos]], mode)) act.push_back((int)pos);
    if (lanes < 2 || (int)act.size() < 2 || mode == M_STRUCT || mode_hess_comp(mode)) return {act};
    // two contiguous subsets, the cut that best balances the outputs (values, first- and
    // second-order slots) of the two sides
    auto cost = [&](int pos) { const Pattern &p = pats[g.pats[pos]]; return 1 + p.nj() + p.nh(); };
    int total = 0;
    for (int pos : act) total += cost(pos);
    int best_cut = 1, best = 1 << 30, left = 0;
    for (size_t c = 1; c < act.size(); c++) {
        left += cost(act[c - 1]);
        const int imbalance = std::abs(2 * left - total);
        if (imbalance < best) { best = imbalance; best_cut = (int)c; }
    }
    return {std::vector<int>(act.begin(), act.begin() + best_cut), std::vector<int>(act.begin() + best_cut, act.end())};
}

namespace {

// ------------------------------------------------------------------ CUDA emission
struct Emitter {
    const std::vector<Pattern> &pats;
    const Group &grp;
    const Graph &g;
    const std::vector<PatternGraph> &PG;  // per position in the group
    const CodegenOptions &opt;
    std::ostringstream os;
    std::string pf_text;  // prefetch functions of the last function() (opt.prefetch > 0)
    // shared-memory staging (opt.stage): the last function()'s stage function and its 8- and
    // 4-byte slot counts per thread
    std::string st_text;
    int n_st8 = 0, n_st4 = 0;
    int st_budget = 0;  // bytes of staged slots one thread may have per buffer (later inputs load from global memory)

    Emitter(const std::vector<Pattern> &p_, const Group &g_, const Graph &gr, const std::vector<PatternGraph> &pg,
            const CodegenOptions &o)
        : pats(p_), grp(g_), g(gr), PG(pg), opt(o) {}

    const Pattern &pat(int pos) const { return pats[grp.pats[pos]]; }

    std::string idx_expr(int pos, int r) {
        const Pattern &p = pat(pos);
        const INode &n = p.ix[r];
        switch (n.op) {
        case EXA_I_CONST: {
            auto it = p.ivary.find(r);
            if (it != p.ivary.end()) return "pm.ic[" + std::to_string(it->second) + "]";
            return "(" + std::to_string(n.iv) + "LL)";
        }
        case EXA_I_FIELD: return "((long long)F" + std::to_string(grp.field[pos][n.iv]) + ")";
        case EXA_I_INST: return "kk";
        default: {
            const char *o = n.op == EXA_I_ADD ? " + " : n.op == EXA_I_SUB ? " - " : " * ";
            return "(" + idx_expr(pos, n.a) + o + idx_expr(pos, n.b) + ")";
        }
        }
    }
    void fields_of_idx(int pos, int r, std::set<int> &f) {
        const INode &n = pat(pos).ix[r];
        if (n.op == EXA_I_FIELD) f.insert(grp.field[pos][n.iv]);
        else if (n.op >= EXA_I_ADD) { fields_of_idx(pos, n.a, f); fields_of_idx(pos, n.b, f); }
    }

    static std::string fname(int op, int prec) {
        const char *n = "?";
        switch (op) {
        case S_EXP: n = "exp"; break; case S_LOG: n = "log"; break; case S_SIN: n = "sin"; break;
        case S_COS: n = "cos"; break; case S_SQRT: n = "sqrt"; break; case S_TAN: n = "tan"; break;
        case S_TANH: n = "tanh"; break; case S_ATAN: n = "atan"; break; case S_SINH: n = "sinh"; break;
        case S_COSH: n = "cosh"; break; case S_ASIN: n = "asin"; break; case S_ACOS: n = "acos"; break;
        case S_LOG1P: n = "log1p"; break; case S_EXPM1: n = "expm1"; break; case S_LOG2: n = "log2"; break;
        case S_LOG10: n = "log10"; break; case S_EXP2: n = "exp2"; break; case S_ATAN2: n = "atan2"; break;
        case S_HYPOT: n = "hypot"; break; case S_POW: n = "pow"; break;
        }
        return std::string(n) + (prec == PF ? "f" : "");
    }
    static const char *ty(int prec) { return prec == PF ? "float" : "double"; }
    static std::string in_name(const SN &s) {
        return std::string(1, s.ikind) + (s.prec == PF ? "F" : "") + std::to_string(s.iid);
    }

    // Emits the nodes the roots need that `name` does not hold yet, in creation (dependency) order,
    // and names them.  sin and cos of one argument are computed together: the pairs are found among
    // the nodes `pair_roots` need (all of a function's roots), so a pair split between two calls
    // is emitted whole at the first.
    void body(const std::vector<int> &roots, std::map<int, std::string> &name,
              const std::vector<int> *pair_roots = nullptr) {
        auto marks = [&](const std::vector<int> &rs) {
            std::vector<char> need(g.n.size(), 0);
            std::function<void(int)> mark = [&](int i) {
                if (need[i]) return;
                need[i] = 1;
                if (g.n[i].a >= 0) mark(g.n[i].a);
                if (g.n[i].b >= 0) mark(g.n[i].b);
            };
            for (int r : rs) mark(r);
            return need;
        };
        const std::vector<char> need = marks(roots);
        const std::vector<char> pneed = pair_roots ? marks(*pair_roots) : need;
        std::map<std::pair<int, int>, std::pair<int, int>> sc;  // (arg, reduced?) -> (sin+1, cos+1)
        for (size_t i = 0; i < g.n.size(); i++) {
            if (!pneed[i]) continue;
            int op = g.n[i].op;
            bool red = op == S_SINR || op == S_COSR;
            if (op == S_SIN || op == S_SINR) sc[{g.n[i].a, red}].first = (int)i + 1;
            if (op == S_COS || op == S_COSR) sc[{g.n[i].a, red}].second = (int)i + 1;
        }
        for (size_t i = 0; i < g.n.size(); i++) {
            if (!need[i] || name.count((int)i)) continue;
            const SN &s = g.n[i];
            const std::string t = "t" + std::to_string(i);
            const char *T = ty(s.prec);
            if (s.op == S_LIT) { name[i] = s.prec == PF ? fmt_float(s.lit) : fmt_double(s.lit); continue; }
            if (s.op == S_IN) { name[i] = in_name(s); continue; }
            name[i] = t;
            auto A = [&]() { return name.at(s.a); };
            auto B = [&]() { return name.at(s.b); };
            switch (s.op) {
            case S_NEG:  // FP64: the sign bit flipped on the integer pipe
                if (s.prec == PD) os << "  const double " << t << " = exa_neg(" << A() << ");\n";
                else os << "  const " << T << " " << t << " = -" << A() << ";\n";
                break;
            case S_ADD: os << "  const " << T << " " << t << " = " << A() << " + " << B() << ";\n"; break;
            case S_SUB: os << "  const " << T << " " << t << " = " << A() << " - " << B() << ";\n"; break;
            case S_MUL:  // FP64 doubling: exact, on the integer pipe
                if (s.prec == PD && (g.is(s.a, 2.0) || g.is(s.b, 2.0)))
                    os << "  const double " << t << " = exa_twice(" << (g.is(s.a, 2.0) ? B() : A()) << ");\n";
                else os << "  const " << T << " " << t << " = " << A() << " * " << B() << ";\n";
                break;
            case S_DIV: os << "  const " << T << " " << t << " = " << A() << " / " << B() << ";\n"; break;
            case S_POW: case S_ATAN2: case S_HYPOT:
                os << "  const " << T << " " << t << " = " << fname(s.op, s.prec) << "(" << A() << ", " << B() << ");\n";
                break;
            case S_CVT:
                if (s.prec == PF) os << "  const float " << t << " = exa_d2f(" << A() << ");\n";
                else os << "  const double " << t << " = exa_f2d(" << A() << ");\n";
                break;
            case S_EXPR: os << "  const float " << t << " = exa_exp_red(" << A() << ");\n"; break;
            case S_SIN: case S_COS: case S_SINR: case S_COSR: {
                bool red = s.op == S_SINR || s.op == S_COSR;
                auto pr = sc[{s.a, red}];
                int si = pr.first - 1, ci = pr.second - 1;
                if (red || (si >= 0 && ci >= 0)) {
                    // the whole pair at its first emitted member; the partner is named here too
                    std::string sn = si >= 0 ? "t" + std::to_string(si) : t + "_s";
                    std::string cn = ci >= 0 ? "t" + std::to_string(ci) : t + "_c";
                    os << "  " << T << " " << sn << ", " << cn << ";\n";
                    if (red) os << "  exa_sincos_red(" << A() << ", &" << sn << ", &" << cn << ");\n";
                    else os << "  " << (s.prec == PF ? "sincosf(" : "exa_sincos64(") << A() << ", &" << sn << ", &" << cn << ");\n";
                    if (si >= 0) name[si] = sn;
                    if (ci >= 0) name[ci] = cn;
                } else if (s.prec == PD) {  // one of the pair: the other result is dead code
                    os << "  double " << t << "_s, " << t << "_c;\n"
                       << "  exa_sincos64(" << A() << ", &" << t << "_s, &" << t << "_c);\n"
                       << "  const double " << t << " = " << t << (s.op == S_SIN ? "_s" : "_c") << ";\n";
                } else {
                    os << "  const " << T << " " << t << " = " << fname(s.op, s.prec) << "(" << A() << ");\n";
                }
                break;
            }
            default: os << "  const " << T << " " << t << " = " << fname(s.op, s.prec) << "(" << A() << ");\n"; break;
            }
        }
    }

    // One device function per (group, mode): every active pattern of the group for one instance.
    // The device function of one warp set (`act`: positions of its patterns; `suffix` names it).
    std::string function(int gid, Mode mode, const std::vector<int> &act, const std::string &suffix = "") {
        os.str("");
        const bool mixed = opt.precision == EXA_MIXED_FP32;
        const char *W = mixed ? "float" : "double";
        const bool all = mode_all(mode) || mode == M_FIRST;
        const bool hs_coo = mode_hess_coo(mode), hs_comp = mode_hess_comp(mode) && !grp.hc.empty();
        const bool want_struct = mode == M_STRUCT;
        // inputs staged in shared memory by the tile loop (s8 / s4: this thread's column of 8- and
        // 4-byte slots of the current buffer, slot j at [j * EXA_BLOCK])
        const bool in_smem = opt.stage && !want_struct && suffix.empty();
        // k is the thread's instance clamped to the last one; act says whether it is its own.  Every
        // lane of a warp runs the function so that outputs can be staged per warp in shared memory
        // (ws) and written back as contiguous, coalesced runs.
        os << "static __device__ __forceinline__ void grp" << gid << "_" << kModeName[mode] << suffix
           << "(const ExaPM& pm, const int k, const bool act, const double* __restrict__ x,"
              " const double* __restrict__ y, const double* __restrict__ th, const double sigma, const ExaOut& o,"
              " const ExaStructOut& so, double& objv, double* __restrict__ ws"
           << (in_smem ? ", const double* __restrict__ s8, const int* __restrict__ s4" : "") << ") {\n";
        os << "  const long long kk = k;\n";
        if (!want_struct)
            os << "  const int lane = threadIdx.x & 31;\n"
                  "  const int nact = __popc(__ballot_sync(0xffffffffu, act));\n"
                  "  const long long kw = __shfl_sync(0xffffffffu, kk, 0);  // instance of lane 0 (active)\n";
        struct Want { bool val, grad, hess, row; };
        std::vector<Want> want(grp.pats.size(), {false, false, false, false});
        std::vector<int> roots;
        std::vector<std::vector<int>> hroots(grp.pats.size());
        for (int pos : act) {
            const Pattern &p = pat(pos);
            const bool obj = p.kind == EXA_OBJ;
            Want &w = want[pos];
            w.val = (mode == M_OBJ && obj) || (mode == M_CON && !obj) || all;
            w.grad = (mode == M_GRAD && obj) || (mode == M_JAC && !obj) || all;
            w.hess = mode_hess(mode) && p.nh() > 0;
            w.row = !obj && (w.val || w.hess || want_struct);
            const PatternGraph &G = PG[pos];
            if (w.val) roots.push_back(G.value);
            if (w.grad) for (int s : p.jsym) roots.push_back(G.grad[s]);
            if (w.hess)
                for (auto &pr : p.hpair) {
                    auto it = G.hess.find({std::min(pr.first, pr.second), std::max(pr.first, pr.second)});
                    hroots[pos].push_back(it == G.hess.end() ? -1 : it->second);
                    if (it != G.hess.end()) roots.push_back(it->second);
                }
        }
        // inputs the roots need, by kind and precision
        std::set<int> syms, fields, params, fconsts;       // FP64 copies (loaded)
        std::set<int> fsyms, ffields, fparams, ffconsts;   // FP32 copies (converted)
        {
            std::vector<char> seen(g.n.size(), 0);
            std::function<void(int)> walk = [&](int i) {
                if (seen[i]) return;
                seen[i] = 1;
                const SN &s = g.n[i];
                if (s.op == S_IN) {
                    std::set<int> *d = s.ikind == 'X' ? &syms : s.ikind == 'D' ? &fields : s.ikind == 'P' ? &params : &fconsts;
                    std::set<int> *f = s.ikind == 'X' ? &fsyms : s.ikind == 'D' ? &ffields : s.ikind == 'P' ? &fparams : &ffconsts;
                    d->insert(s.iid);
                    if (s.prec == PF) f->insert(s.iid);
                }
                if (s.a >= 0) walk(s.a);
                if (s.b >= 0) walk(s.b);
            };
            for (int r : roots) walk(r);
        }
        std::set<int> idx_syms = syms;  // group symbols whose index is needed
        for (int pos : act) {
            const Pattern &p = pat(pos);
            if (want_struct) for (int s = 0; s < p.nsym; s++) idx_syms.insert(grp.sym[pos][s]);
            if (want[pos].hess)
                for (auto &pr : p.hpair)
                    if (pr.first != pr.second) { idx_syms.insert(grp.sym[pos][pr.first]); idx_syms.insert(grp.sym[pos][pr.second]); }
        }
        // columns used as FP64 values (D) and as FP32 values (DF); in mixed mode f64 columns have an
        // FP32 copy (pm.f32) that FP32 uses load directly
        std::set<int> dfields, fcopy;
        {
            std::vector<char> seen(g.n.size(), 0);
            std::function<void(int)> walk = [&](int i) {
                if (seen[i]) return;
                seen[i] = 1;
                const SN &sn = g.n[i];
                if (sn.op == S_IN && sn.ikind == 'D') {
                    if (sn.prec == PD) dfields.insert(sn.iid);
                    else if (grp.ftype[sn.iid] == EXA_FIELD_F64) fcopy.insert(sn.iid);
                    else dfields.insert(sn.iid);  // int32 column used as an FP32 value: convert the int
                }
                if (sn.a >= 0) walk(sn.a);
                if (sn.b >= 0) walk(sn.b);
            };
            for (int r : roots) walk(r);
        }
        std::set<int> all_fields = dfields;
        for (int s : idx_syms) fields_of_idx(grp.sym_root[s].first, grp.sym_root[s].second, all_fields);
        for (int pid : params) fields_of_idx(pid / 65536, pat(pid / 65536).v[pid % 65536].a, all_fields);
        for (int pos : act)
            if (want[pos].row && pat(pos).kind == EXA_AUG) fields_of_idx(pos, pat(pos).row_root, all_fields);
        const bool lazy = opt.by_pattern && opt.lazy_loads && !want_struct;
        // Staged inputs: every data column, the FP32 column copies, the x values whose index is
        // the instance plus constants, and the multipliers of constraint rows; the tile loop copies
        // them for the CTA's next tile (cp.async) while this tile computes.  Gathers through data
        // fields are loaded here from global memory, their index fields coming from shared memory.
        std::map<std::string, int> st8, st4;
        std::vector<std::string> st_src8, st_src4;
        if (in_smem) {
            int bytes = 0;
            auto add = [&](std::map<std::string, int> &mp, std::vector<std::string> &src, const std::string &key,
                           const std::string &addr) {
                const int b = &mp == &st8 ? 8 : 4;
                if (mp.count(key) || bytes + b > st_budget) return;
                bytes += b;
                mp.emplace(key, (int)src.size());
                src.push_back(addr);
            };
            for (int f : all_fields) {
                const std::string F = std::to_string(f);
                if (grp.ftype[f] == EXA_FIELD_I32) add(st4, st_src4, "F" + F, "(const int*)pm.f[" + F + "] + k");
                else add(st8, st_src8, "F" + F, "(const double*)pm.f[" + F + "] + k");
            }
            for (int f : fcopy) add(st4, st_src4, "DF" + std::to_string(f), "pm.f32[" + std::to_string(f) + "] + k");
            for (int sy : syms) {
                std::set<int> fs;
                fields_of_idx(grp.sym_root[sy].first, grp.sym_root[sy].second, fs);
                if (fs.empty())
                    add(st8, st_src8, "X" + std::to_string(sy),
                        "x + pm.xoff + " + idx_expr(grp.sym_root[sy].first, grp.sym_root[sy].second));
            }
            for (int pos : act)
                if (want[pos].hess && pat(pos).kind == EXA_CON)
                    add(st8, st_src8, "Y" + std::to_string(pos), "y + pm.rbase[" + std::to_string(pos) + "] + kk");
        }
        // the load of one input: its shared-memory slot when staged, else global memory
        auto ld = [&](const std::string &key, const std::string &global) -> std::string {
            auto i8 = st8.find(key);
            if (i8 != st8.end()) return "s8[" + std::to_string(i8->second) + " * EXA_BLOCK]";
            auto i4 = st4.find(key);
            if (i4 != st4.end())
                return key[0] == 'D' ? "__int_as_float(s4[" + std::to_string(i4->second) + " * EXA_BLOCK])"
                                     : "s4[" + std::to_string(i4->second) + " * EXA_BLOCK]";
            return "__ldg(" + global + ")";
        };
        st_text.clear();
        n_st8 = (int)st_src8.size();
        n_st4 = (int)st_src4.size();
        if (in_smem && (n_st8 + n_st4) > 0) {
            std::ostringstream st;
            st << "static __device__ __forceinline__ void grp" << gid << "_" << kModeName[mode]
               << "_st(const ExaPM& pm, const int k, const double* __restrict__ x, const double* __restrict__ y,"
                  " const unsigned d8, const unsigned d4) {\n"
                  "  const long long kk = k;\n";
            for (size_t j = 0; j < st_src8.size(); j++)
                st << "  exa_cp_async8(d8 + " << j << "u * (EXA_BLOCK * 8u), " << st_src8[j] << ");\n";
            for (size_t j = 0; j < st_src4.size(); j++)
                st << "  exa_cp_async4(d4 + " << j << "u * (EXA_BLOCK * 4u), " << st_src4[j] << ");\n";
            st << "}\n";
            st_text = st.str();
        }
        for (int f : all_fields) {
            const std::string F = std::to_string(f);
            if (grp.ftype[f] == EXA_FIELD_I32)
                os << "  const int F" << f << " = " << ld("F" + F, "(const int*)pm.f[" + F + "] + k") << ";\n";
            else if (!lazy)
                os << "  const double F" << f << " = " << ld("F" + F, "(const double*)pm.f[" + F + "] + k") << ";\n";
        }
        if (!lazy) {
            for (int f : dfields)
                os << "  const double D" << f << " = " << (grp.ftype[f] == EXA_FIELD_I32 ? "(double)F" : "F") << f << ";\n";
            for (int f : fcopy)
                os << "  const float DF" << f << " = " << ld("DF" + std::to_string(f), "pm.f32[" + std::to_string(f) + "] + k") << ";\n";
        }
        for (int s : idx_syms) {
            os << "  long long i" << s << " = " << idx_expr(grp.sym_root[s].first, grp.sym_root[s].second) << ";\n";
            if (opt.bounds_check || want_struct)
                os << "  if ((unsigned long long)i" << s << " >= (unsigned long long)pm.nvar_m) { atomicOr(o.status, 1); i" << s << " = 0; }\n";
        }
        for (int pid : params) {
            int pos = pid / 65536, node = pid % 65536;
            os << "  long long q" << pid << " = " << idx_expr(pos, pat(pos).v[node].a) << ";\n";
            if (opt.bounds_check || want_struct)
                os << "  if ((unsigned long long)q" << pid << " >= (unsigned long long)pm.npar_m) { atomicOr(o.status, 1); q" << pid << " = 0; }\n";
        }
        for (int pos : act) {
            if (!want[pos].row) continue;
            const Pattern &p = pat(pos);
            if (p.kind == EXA_CON) os << "  const long long row" << pos << " = pm.rbase[" << pos << "] + kk;\n";
            else {
                os << "  long long lrow" << pos << " = " << idx_expr(pos, p.row_root) << ";\n";
                if (opt.bounds_check || want_struct)
                    os << "  if ((unsigned long long)lrow" << pos << " >= (unsigned long long)pm.rlimit[" << pos
                       << "]) { atomicOr(o.status, 1); lrow" << pos << " = 0; }\n";
                os << "  const long long row" << pos << " = pm.rbase[" << pos << "] + lrow" << pos << ";\n";
            }
        }
        pf_text.clear();
        if (!want_struct && opt.prefetch > 0) {
            // _pf: lane c of a warp prefetches data column c of the tile starting at `begin` into L2
            // (one bulk prefetch per column; 16-byte aligned since begin is a multiple of the
            // block and columns are cudaMalloc'd; the size is rounded down, so it stays in bounds)
            std::ostringstream pf;
            pf << "static __device__ __forceinline__ void grp" << gid << "_" << kModeName[mode]
               << "_pf(const ExaPM& pm, const int begin) {\n"
                  "  const long long n = pm.n_inst - begin < EXA_BLOCK ? pm.n_inst - begin : EXA_BLOCK;\n"
                  "  const void* p = nullptr;\n  int es = 0;\n  switch (threadIdx.x & 31) {\n";
            int lane_no = 0;
            for (int f : all_fields)
                pf << "    case " << lane_no++ << ": p = pm.f[" << f << "]; es = "
                   << (grp.ftype[f] == EXA_FIELD_I32 ? 4 : 8) << "; break;\n";
            for (int f : fcopy) pf << "    case " << lane_no++ << ": p = pm.f32[" << f << "]; es = 4; break;\n";
            pf << "    default: return;\n  }\n"
                  "  const unsigned bytes = (unsigned)(n * es) & ~15u;\n"
                  "  if (bytes) asm volatile(\"cp.async.bulk.prefetch.L2.global [%0], %1;\" :: \"l\"((const char*)p + (long long)begin * es), \"r\"(bytes) : \"memory\");\n"
                  "}\n";
            // _pfx: the x and y lines instance k gathers, prefetched into L2 (indices were checked
            // by the structure pass at creation, so every address is inside x or y)
            pf << "static __device__ __forceinline__ void grp" << gid << "_" << kModeName[mode]
               << "_pfx(const ExaPM& pm, const int k, const double* __restrict__ x, const double* __restrict__ y) {\n"
                  "  const long long kk = k;\n";
            std::set<int> ixf;
            for (int sy : syms) fields_of_idx(grp.sym_root[sy].first, grp.sym_root[sy].second, ixf);
            std::vector<int> yrows;
            for (int pos : act)
                if (want[pos].hess && pat(pos).kind != EXA_OBJ) {
                    yrows.push_back(pos);
                    if (pat(pos).kind == EXA_AUG) fields_of_idx(pos, pat(pos).row_root, ixf);
                }
            for (int f : ixf)
                pf << "  const int F" << f << " = __ldg((const int*)pm.f[" << f << "] + k);\n";
            for (int sy : syms)
                pf << "  asm volatile(\"prefetch.global.L2 [%0];\" :: \"l\"(x + pm.xoff + "
                   << idx_expr(grp.sym_root[sy].first, grp.sym_root[sy].second) << "));\n";
            for (int pos : yrows) {
                const std::string row = pat(pos).kind == EXA_CON
                                            ? "pm.rbase[" + std::to_string(pos) + "] + kk"
                                            : "pm.rbase[" + std::to_string(pos) + "] + " + idx_expr(pos, pat(pos).row_root);
                pf << "  asm volatile(\"prefetch.global.L2 [%0];\" :: \"l\"(y + " << row << "));\n";
            }
            pf << "}\n";
            pf_text = pf.str();
        }
        if (want_struct) {
            os << "  if (!act) return;\n";
            for (int pos : act) {
                const Pattern &p = pat(pos);
                const std::string P = std::to_string(pos);
                auto gs = [&](int s) { return "i" + std::to_string(grp.sym[pos][s]); };
                if (p.kind == EXA_OBJ) {
                    for (int j = 0; j < p.nj(); j++)
                        os << "  so.gvar[pm.gbase[" << P << "] + kk * " << p.nj() << " + " << j << "] = (int)(pm.xoff + " << gs(p.jsym[j]) << ");\n";
                } else {
                    for (int j = 0; j < p.nj(); j++) {
                        os << "  so.jrow[pm.jbase[" << P << "] + kk * " << p.nj() << " + " << j << "] = (int)row" << P << ";\n";
                        os << "  so.jcol[pm.jbase[" << P << "] + kk * " << p.nj() << " + " << j << "] = (int)(pm.xoff + " << gs(p.jsym[j]) << ");\n";
                    }
                    if (p.kind == EXA_AUG) os << "  so.arow[pm.abase[" << P << "] + kk] = (int)row" << P << ";\n";
                }
                for (int j = 0; j < p.nh(); j++) {
                    int a = p.hpair[j].first, b = p.hpair[j].second;
                    os << "  { const long long ga = pm.xoff + " << gs(a) << ", gb = pm.xoff + " << gs(b) << ";\n"
                       << "    so.hrow[pm.hbase[" << P << "] + kk * " << p.nh() << " + " << j << "] = (int)(ga > gb ? ga : gb);\n"
                       << "    so.hcol[pm.hbase[" << P << "] + kk * " << p.nh() << " + " << j << "] = (int)(ga > gb ? gb : ga); }\n";
                }
            }
            const int nhc = (int)grp.hc.size();
            if (nhc > 0) {
                os << "  if (so.hcrow) {\n";
                for (int c = 0; c < nhc; c++)
                    os << "    { const long long ga = pm.xoff + i" << grp.hc_sym[c].first << ", gb = pm.xoff + i"
                       << grp.hc_sym[c].second << ";\n"
                       << "      so.hcrow[pm.hcbase + kk * " << nhc << " + " << c << "] = (int)(ga > gb ? ga : gb);\n"
                       << "      so.hccol[pm.hcbase + kk * " << nhc << " + " << c << "] = (int)(ga > gb ? gb : ga); }\n";
                os << "  }\n";
            }
            os << "}\n";
            return os.str();
        }
        if (!lazy)
            for (int s : syms)
                os << "  const double X" << s << " = " << ld("X" + std::to_string(s), "x + pm.xoff + i" + std::to_string(s)) << ";\n";
        // Pairs of different symbols whose slot doubles when both resolve to one variable: their
        // equality tests are taken once here, into one bit mask, so that the 64-bit indices are
        // dead once the gathers are issued instead of staying live until the Hessian.
        std::map<std::pair<int, int>, int> eqbit;
        for (int pos : act)
            if (want[pos].hess)
                for (auto &pr : pat(pos).hpair)
                    if (pr.first != pr.second) {
                        int ga = grp.sym[pos][pr.first], gb = grp.sym[pos][pr.second];
                        eqbit.emplace(std::make_pair(std::min(ga, gb), std::max(ga, gb)), (int)eqbit.size());
                    }
        const bool use_eqm = !eqbit.empty() && eqbit.size() <= 64;
        if (use_eqm) {
            os << "  const unsigned long long eqm = 0ull";
            for (auto &kv : eqbit)
                os << " | ((unsigned long long)(i" << kv.first.first << " == i" << kv.first.second << ") << " << kv.second
                   << ")";
            os << ";\n";
        }
        for (int c : fconsts) os << "  const double C" << c << " = pm.fc[" << c << "];\n";
        for (int c : ffconsts) os << "  const float CF" << c << " = exa_d2f(C" << c << ");\n";
        // Inputs of the patterns: loads issued (`issue`) and FP32 copies formed (`ready`).  Eagerly:
        // everything at the top.  Lazily: a pattern's loads are issued before the arithmetic of the
        // pattern preceding it (one pattern of lookahead covers their latency), and its FP32
        // copies are formed where its own arithmetic starts.
        std::set<std::string> issued, readied;
        auto issue_in = [&](const SN &sn) {
            const std::string key = std::string(1, sn.ikind) + std::to_string(sn.iid);
            if (!issued.insert(key).second) return;
            switch (sn.ikind) {
            case 'X':
                os << "  const double X" << sn.iid << " = " << ld("X" + std::to_string(sn.iid), "x + pm.xoff + i" + std::to_string(sn.iid)) << ";\n";
                break;
            case 'P': os << "  const double P" << sn.iid << " = __ldg(th + pm.poff + q" << sn.iid << ");\n"; break;
            case 'D':
                if (grp.ftype[sn.iid] == EXA_FIELD_F64) {
                    if (dfields.count(sn.iid) || (sn.prec == PD))
                        os << "  const double F" << sn.iid << " = "
                           << ld("F" + std::to_string(sn.iid), "(const double*)pm.f[" + std::to_string(sn.iid) + "] + k") << ";\n"
                           << "  const double D" << sn.iid << " = F" << sn.iid << ";\n";
                    if (fcopy.count(sn.iid))
                        os << "  const float DF" << sn.iid << " = "
                           << ld("DF" + std::to_string(sn.iid), "pm.f32[" + std::to_string(sn.iid) + "] + k") << ";\n";
                }
                break;
            default: break;
            }
        };
        auto ready_in = [&](const SN &sn) {
            const std::string key = std::string(1, sn.ikind) + std::to_string(sn.iid) + (sn.prec == PF ? "f" : "d");
            if (!readied.insert(key).second) return;
            if (sn.ikind == 'X' && sn.prec == PF) os << "  const float XF" << sn.iid << " = exa_d2f(X" << sn.iid << ");\n";
            if (sn.ikind == 'P' && sn.prec == PF) os << "  const float PF" << sn.iid << " = exa_d2f(P" << sn.iid << ");\n";
            if (sn.ikind == 'D' && grp.ftype[sn.iid] == EXA_FIELD_I32) {
                if (sn.prec == PF) os << "  const float DF" << sn.iid << " = (float)F" << sn.iid << ";\n";
                else os << "  const double D" << sn.iid << " = (double)F" << sn.iid << ";\n";
            }
        };
        // inputs of every pattern, from its roots
        std::map<int, std::vector<int>> pin;  // position -> S_IN nodes
        {
            for (int pos : act) {
                std::vector<int> rs;
                const PatternGraph &G = PG[pos];
                if (want[pos].val) rs.push_back(G.value);
                if (want[pos].grad) for (int sy : pat(pos).jsym) rs.push_back(G.grad[sy]);
                for (int r : hroots[pos]) if (r >= 0) rs.push_back(r);
                std::vector<char> seen(g.n.size(), 0);
                std::function<void(int)> walk = [&](int i) {
                    if (seen[i]) return;
                    seen[i] = 1;
                    if (g.n[i].op == S_IN && g.n[i].ikind != 'C') pin[pos].push_back(i);
                    if (g.n[i].a >= 0) walk(g.n[i].a);
                    if (g.n[i].b >= 0) walk(g.n[i].b);
                };
                for (int r : rs) walk(r);
            }
        }
        auto issue_pattern = [&](int pos) {
            for (int i : pin[pos]) issue_in(g.n[i]);
            if (want[pos].hess && pat(pos).kind != EXA_OBJ && issued.insert("Y" + std::to_string(pos)).second)
                os << "  const double Y" << pos << " = " << ld("Y" + std::to_string(pos), "y + row" + std::to_string(pos)) << ";\n";
        };
        auto ready_pattern = [&](int pos) { for (int i : pin[pos]) ready_in(g.n[i]); };
        if (!lazy) {
            for (int pid : params) os << "  const double P" << pid << " = __ldg(th + pm.poff + q" << pid << ");\n";
            // the multipliers of the constraint rows are loaded with the other inputs, so that their
            // latency overlaps the pattern arithmetic instead of following it
            for (int pos : act)
                if (want[pos].hess && pat(pos).kind != EXA_OBJ)
                    os << "  const double Y" << pos << " = " << ld("Y" + std::to_string(pos), "y + row" + std::to_string(pos)) << ";\n";
            for (int s : fsyms) os << "  const float XF" << s << " = exa_d2f(X" << s << ");\n";
            for (int f : ffields)
                if (!fcopy.count(f)) os << "  const float DF" << f << " = (float)F" << f << ";\n";  // int32 column
            for (int pid : fparams) os << "  const float PF" << pid << " = exa_d2f(P" << pid << ");\n";
        } else if (!act.empty()) {
            issue_pattern(act[0]);
            if (act.size() > 1) issue_pattern(act[1]);
        }
        std::map<int, std::string> name;
        if (!opt.by_pattern) body(roots, name);
        auto widen = [&](int r) { return g.n[r].prec == PF ? "exa_f2d(" + name.at(r) + ")" : name.at(r); };
        // csc/map: optional direct CSC output (a pure permutation of the COO slots); out/slot are
        // the COO array and the block's first slot
        auto staged = [&](const std::string &out, const std::string &slot0, int S, const std::vector<std::string> &vals,
                          const char *csc, const char *map) {
            os << "  __syncwarp();\n";
            for (int j = 0; j < S; j++) os << "  ws[lane * " << S << " + " << j << "] = " << vals[j] << ";\n";
            // a full warp writes S x 32 consecutive values: unrolled, one address computation
            os << "  __syncwarp();\n"
               << "  { const long long q0 = " << slot0 << " + kw * " << S << ";\n"
               << "    if (" << out << ") {\n"
               << "      if (nact == 32) { double* __restrict__ d = " << out << " + q0 + lane;\n"
               << "        #pragma unroll\n"
               << "        for (int j = 0; j < " << S << "; j++) d[32 * j] = ws[lane + 32 * j]; }\n"
               << "      else for (int e = lane; e < nact * " << S << "; e += 32) " << out << "[q0 + e] = ws[e];\n"
               << "    }\n";
            if (csc)
                os << "    if (" << csc << ") for (int e = lane; e < nact * " << S << "; e += 32) "
                   << csc << "[" << map << "[q0 + e]] = ws[e];\n";
            os << "  }\n";
        };
        std::map<std::pair<int, int>, int> hc_of;  // (position, slot) -> compressed slot
        for (size_t c = 0; c < grp.hc.size(); c++)
            for (auto &pj : grp.hc[c]) hc_of[pj] = (int)c;
        std::vector<char> hc_started(grp.hc.size(), 0);
        // Compressed sums, from the slots' products before any doubling.  Each sum is a sequence of
        // terms (pattern, product node, sign; a slot whose two different symbols are one group
        // symbol always holds twice its product).  Two sums whose sequences agree up to one overall
        // sign are equal up to that sign, bit for bit (same operands added in the same order), so
        // the later one is the earlier one negated or copied: the angle-difference patterns of power
        // flow give h(tf,tf) = h(tt,tt) = -h(tf,tt), and likewise for their mixed partials.  A sum
        // over two different symbols is doubled afterwards, as a whole, where they resolve to one
        // variable (2 a + 2 b = 2 (a + b) exactly).
        std::vector<int> hc_dup(grp.hc.size(), -1), hc_dsign(grp.hc.size(), 1);
        std::vector<std::vector<char>> hc_twice(grp.hc.size());  // per term of hc[c]: always doubled
        if (hs_comp) {
            std::map<std::vector<long long>, std::pair<int, int>> seen;  // normalised terms -> (sum, sign)
            for (size_t c = 0; c < grp.hc.size(); c++) {
                std::vector<long long> key;
                int first_sign = 0;
                hc_twice[c].assign(grp.hc[c].size(), 0);
                for (size_t t = 0; t < grp.hc[c].size(); t++) {
                    const int pos = grp.hc[c][t].first, j = grp.hc[c][t].second;
                    if (std::find(act.begin(), act.end(), pos) == act.end() || !want[pos].hess) continue;
                    const Pattern &p = pat(pos);
                    const int a = p.hpair[j].first, b = p.hpair[j].second;
                    const bool twice = a != b && grp.sym[pos][a] == grp.sym[pos][b];
                    hc_twice[c][t] = twice;
                    const int r = hroots[pos][j];
                    int base = -1, sign = 1;
                    if (r >= 0) {
                        const bool ng = g.n[r].op == S_NEG;
                        base = ng ? g.n[r].a : r;
                        sign = ng ? -1 : 1;
                    }
                    if (!first_sign) first_sign = sign;
                    key.push_back(((long long)pos << 40) ^ ((long long)(base + 1) << 2) ^ (twice ? 2 : 0) ^
                                  (sign * first_sign < 0 ? 1 : 0));
                }
                if (key.empty()) continue;
                auto it = seen.find(key);
                if (it == seen.end()) seen.emplace(key, std::make_pair((int)c, first_sign));
                else {
                    hc_dup[c] = it->second.first;
                    hc_dsign[c] = first_sign * it->second.second;
                }
            }
        }
        for (int pos : act) {
            const Pattern &p = pat(pos);
            const PatternGraph &G = PG[pos];
            const Want &w = want[pos];
            const std::string P = std::to_string(pos);
            const bool obj = p.kind == EXA_OBJ;
            if (lazy) {  // this pattern's FP32 copies; the next pattern's loads
                const size_t j = std::find(act.begin(), act.end(), pos) - act.begin();
                ready_pattern(pos);
                if (j + 2 <= act.size() && j + 1 < act.size()) issue_pattern(act[j + 1]);
            }
            if (opt.by_pattern) {  // this pattern's arithmetic, right before its outputs
                std::vector<int> mine;
                if (w.val) mine.push_back(G.value);
                if (w.grad) for (int sy : p.jsym) mine.push_back(G.grad[sy]);
                for (int r : hroots[pos]) if (r >= 0) mine.push_back(r);
                body(mine, name, &roots);
            }
            if (w.val) {
                const std::string v = widen(G.value);
                if (obj) os << "  if (act) objv += " << v << ";\n";  // the thread's running objective sum
                else if (p.kind == EXA_CON) os << "  if (act) o.c[row" << P << "] = " << v << ";\n";
                else os << "  if (act) o.abuf[pm.abase[" << P << "] + kk] = " << v << ";\n";
            }
            // a block of S slots per instance: stage the warp's 32 x S values, then write the warp's
            // contiguous run of nact x S values with consecutive lanes on consecutive addresses
            if (w.grad && p.nj() > 0) {
                std::vector<std::string> vals;
                for (int j = 0; j < p.nj(); j++) vals.push_back(widen(G.grad[p.jsym[j]]));
                if (obj) staged("o.gbuf", "pm.gbase[" + P + "]", p.nj(), vals, nullptr, nullptr);
                else staged("o.jac", "pm.jbase[" + P + "]", p.nj(), vals, "o.jcsc", "o.jmap");
            }
            if (w.hess) {
                os << "  const " << W << " w" << P << " = " << (obj ? (mixed ? "exa_d2f(sigma)" : "sigma")
                                                          : (mixed ? "exa_d2f(Y" + P + ")" : "Y" + P))
                   << ";\n";
                // The weight multiplies each distinct second partial once: slots whose values differ
                // only in sign share one product.
                std::map<int, std::string> prod;
                std::vector<std::string> vals;
                std::string coll;  // some symbol pair of this pattern resolves to one variable
                std::vector<std::pair<int, std::string>> doubled;
                for (int j = 0; j < p.nh(); j++) {
                    const int a = p.hpair[j].first, b = p.hpair[j].second;
                    const int r = hroots[pos][j];
                    const std::string hv = "hv" + P + "_" + std::to_string(j);
                    std::string v = "0.0";
                    if (r >= 0) {
                        const bool ng = g.n[r].op == S_NEG;
                        const int base = ng ? g.n[r].a : r;
                        auto it = prod.find(base);
                        if (it == prod.end()) {
                            const std::string pn = "hp" + P + "_" + std::to_string(prod.size());
                            if (!mixed && g.is(base, 2.0))
                                os << "  const double " << pn << " = exa_twice(w" << P << ");\n";
                            else
                                os << "  const " << W << " " << pn << " = w" << P << " * " << name.at(base) << ";\n";
                            it = prod.emplace(base, pn).first;
                        }
                        v = mixed ? "exa_f2d(" + std::string(ng ? "-" : "") + it->second + ")"
                                  : (ng ? "exa_neg(" + it->second + ")" : it->second);
                    }
                    os << "  double " << hv << " = " << v << ";\n";
                    vals.push_back(hv);
                    if (a != b) {
                        const int ga = grp.sym[pos][a], gb = grp.sym[pos][b];
                        const std::string c =
                            use_eqm ? "((eqm >> " + std::to_string(eqbit.at({std::min(ga, gb), std::max(ga, gb)})) + ") & 1ull)"
                                    : "(i" + std::to_string(ga) + " == i" + std::to_string(gb) + ")";
                        coll += (coll.empty() ? "" : " || ") + c;
                        doubled.push_back({j, c});
                    }
                }
                if (hs_comp)  // the group's compressed sums (FP64, pattern order), before the doubling
                    for (int j = 0; j < p.nh(); j++) {
                        const int c = hc_of.at({pos, j});
                        if (hc_dup[c] >= 0) continue;  // equal up to sign to an earlier sum
                        size_t t = 0;
                        while (grp.hc[c][t] != std::make_pair(pos, j)) t++;
                        const std::string term = hc_twice[c][t] ? "exa_twice(" + vals[j] + ")" : vals[j];
                        if (hc_started[c]) os << "  hc" << c << " += " << term << ";\n";
                        else os << "  double hc" << c << " = " << term << ";\n";
                        hc_started[c] = 1;
                    }
                // A slot pairing two different symbols that resolve to the same variable holds twice
                // the mixed partial (2 (w h) equals (2 w) h exactly).  Rare: one warp-uniform test,
                // the doubling only in warps that need it.
                if (!doubled.empty()) {
                    os << "  if (__any_sync(0xffffffffu, " << coll << ")) {\n";
                    for (auto &dj : doubled)
                        os << "    if (" << dj.second << ") hv" << P << "_" << dj.first << " += hv" << P << "_"
                           << dj.first << ";\n";
                    os << "  }\n";
                }
                if (hs_coo) staged("o.hess", "pm.hbase[" + P + "]", p.nh(), vals, "o.hcsc", "o.hmap");
            }
        }
        if (hs_comp) {  // per-instance FP64 sums of the Hessian slots that share (row, col) in the group
            for (size_t c = 0; c < grp.hc.size(); c++)
                if (hc_dup[c] >= 0 && hc_started[hc_dup[c]]) {
                    const std::string src = "hc" + std::to_string(hc_dup[c]);
                    os << "  double hc" << c << " = " << (hc_dsign[c] < 0 ? "exa_neg(" + src + ")" : src) << ";\n";
                    hc_started[c] = 1;
                }
            // sums over two different symbols that resolve to one variable: doubled as a whole
            std::string any;
            std::vector<std::pair<size_t, std::string>> dbl;
            for (size_t c = 0; c < grp.hc.size(); c++) {
                const int ga = grp.hc_sym[c].first, gb = grp.hc_sym[c].second;
                if (!hc_started[c] || ga == gb) continue;
                auto eb = eqbit.find({std::min(ga, gb), std::max(ga, gb)});
                const std::string cond = use_eqm && eb != eqbit.end()
                                             ? "((eqm >> " + std::to_string(eb->second) + ") & 1ull)"
                                             : "(i" + std::to_string(ga) + " == i" + std::to_string(gb) + ")";
                any += (any.empty() ? "" : " || ") + cond;
                dbl.push_back({c, cond});
            }
            if (!dbl.empty()) {
                os << "  if (__any_sync(0xffffffffu, " << any << ")) {\n";
                for (auto &d : dbl) os << "    if (" << d.second << ") hc" << d.first << " += hc" << d.first << ";\n";
                os << "  }\n";
            }
            std::vector<std::string> sums;
            for (size_t c = 0; c < grp.hc.size(); c++) sums.push_back(hc_started[c] ? "hc" + std::to_string(c) : "0.0");
            staged("o.hcomp", "pm.hcbase", (int)grp.hc.size(), sums, nullptr, nullptr);
        }
        os << "}\n";
        return os.str();
    }
};

// Mixed-mode helpers.  Cody-Waite reduction (Cody & Waite, 1980) in FP64 with a two-part constant:
// the high part carries 32 significant bits, so q * HI is exact for |q| < 2^21 and r = a - q*HI - q*LO
// is accurate to about 1e-16 |a|; the reduced argument is then rounded to FP32 and passed to the
// single-precision functions.  Outside the exact range the FP64 function is used.
// PIO2_HI / PIO2_LO: pi/2 rounded to 32 bits and the rounded remainder; LN2_HI / LN2_LO likewise
// for ln 2 (computed with 300-bit arithmetic).
// FP32 <-> FP64 conversions done with integer operations (the IEEE-754 encodings, round to nearest
// even), exact for every value whose result is a normal number or zero; the remaining cases
// (subnormal results, infinities, NaN) take the hardware conversion.  On GB300 the hardware
// conversions issue on the narrow FP64 pipe, the integer ops do not.
static const char *kMixedHelpers = R"(
static __device__ __forceinline__ double exa_f2d(const float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u < 254u)
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu)), (int)(u << 29));
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}
static __device__ __forceinline__ float exa_d2f(const double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    const unsigned bits = (hi & 0x80000000u) | ((e - 896u) << 23) | m;
    return __uint_as_float(bits + ((rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u))));
  }
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return (float)d;
}
)"
R"(
static __device__ __forceinline__ void exa_sincos_red(const double a, float* s, float* c) {
  if (!(fabs(a) < 1.0e6)) { double sd, cd; sincos(a, &sd, &cd); *s = (float)sd; *c = (float)cd; return; }
  const double q = rint(a * 0x1.45f306dc9c883p-1);
  const double r = fma(-q, 0x1.0b4611a626331p-34, fma(-q, 0x1.921fb54400000p+0, a));
  float sr, cr;
  sincosf(exa_d2f(r), &sr, &cr);
  switch (((int)q) & 3) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}
static __device__ __forceinline__ float exa_exp_red(const double a) {
  if (!(fabs(a) < 80.0)) return (float)exp(a);
  const double k = rint(a * 0x1.71547652b82fep+0);
  const double r = fma(-k, -0x1.718432a1b0e26p-35, fma(-k, 0x1.62e42ff000000p-1, a));
  return ldexpf(expf(exa_d2f(r)), (int)k);
}
)";

// Exact FP64 operations on the integer pipe.  GB300's FP64 pipe retires two operations per clock
// per SM, its integer pipes sixty-four: a negation or a doubling done with the bits of the value
// costs a few integer operations instead of a slot on the binding unit.
//   exa_neg:   IEEE negation is the sign bit flipped (NaN included).
//   exa_twice: 2 v: a normal v below the largest binade gets its exponent increased by one; zeros
//              and subnormals have their magnitude bits shifted left once (a carry into the exponent
//              field gives the right normal number); the largest binade overflows to infinity with
//              v's sign; infinities and NaN are returned unchanged.
static const char *kExactHelpers = R"(
static __device__ __forceinline__ double exa_neg(const double v) {
  return __hiloint2double(__double2hiint(v) ^ (int)0x80000000u, __double2loint(v));
}
static __device__ __forceinline__ double exa_twice(const double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned e = (hi >> 20) & 0x7ffu, sg = hi & 0x80000000u;
  unsigned nh = hi, nl = lo;
  if (e - 1u < 0x7fdu) nh = hi + 0x100000u;
  else if (e == 0u) { nh = sg | ((hi << 1) & 0x7fffffffu) | (lo >> 31); nl = lo << 1; }
  else if (e == 0x7feu) { nh = sg | 0x7ff00000u; nl = 0u; }
  return __hiloint2double((int)nh, (int)nl);
}
)";

// FP64 sin/cos helper of the generated code (its own file, so that a host test can compile it)
static const char *kFp64Helpers =
#include "exa_fp64_sincos.inc"
    ;

// Reductions of the fused step (ExaRed), run by one CTA over [p0, p1).  Values written by other
// CTAs during the kernel (COO slots, compressed sums, gradient and augmentation buffers,
// constraint base values) are read through L2 (ld.global.cg); the index arrays are constant.
// Each segment is added in ascending order starting from its first entry (how 1), from 0.0 (how 2)
// or from dst[rows[s]] (how 3): the additions of the two-pass CSC sums and of the segment kernels.
static const char *kStepHelpers = R"(
static __device__ __forceinline__ void exa_red_perm(const ExaRed& r, const int p0, const int p1) {
  for (int base = p0 + (int)threadIdx.x; base < p1; base += EXA_BLOCK * 8) {
    int q[8];
    #pragma unroll
    for (int u = 0; u < 8; u++) { const int p = base + u * EXA_BLOCK; q[u] = p < p1 ? __ldg(r.perm + p) : -1; }
    double v[8];
    #pragma unroll
    for (int u = 0; u < 8; u++) v[u] = q[u] >= 0 ? __ldcg(r.src + q[u]) : 0.0;
    #pragma unroll
    for (int u = 0; u < 8; u++) if (q[u] >= 0) r.dst[base + u * EXA_BLOCK] = v[u];
  }
}
static __device__ __forceinline__ void exa_red_seg(const ExaRed& r, const int p0, const int p1) {
  for (int base = p0 + (int)threadIdx.x; base < p1; base += EXA_BLOCK * 4) {
    int b[4], e[4], q0[4];
    long long d[4];
    double acc[4];
    #pragma unroll
    for (int u = 0; u < 4; u++) {
      const int s = base + u * EXA_BLOCK;
      b[u] = s < p1 ? __ldg(r.ptr + s) : 0;
      e[u] = s < p1 ? __ldg(r.ptr + s + 1) : 0;
      d[u] = r.how == 3 && s < p1 ? (long long)__ldg(r.rows + s) : (long long)s;
    }
    #pragma unroll
    for (int u = 0; u < 4; u++) {
      q0[u] = b[u] < e[u] ? __ldg(r.perm + b[u]) : -1;
      acc[u] = r.how == 3 && base + u * EXA_BLOCK < p1 ? __ldcg(r.dst + d[u]) : 0.0;
    }
    #pragma unroll
    for (int u = 0; u < 4; u++)
      if (q0[u] >= 0) { const double v = __ldcg(r.src + q0[u]); acc[u] = r.how == 1 ? v : acc[u] + v; }
    #pragma unroll
    for (int u = 0; u < 4; u++) {
      for (int q = b[u] + 1; q < e[u]; q++) acc[u] += __ldcg(r.src + __ldg(r.perm + q));
      if (base + u * EXA_BLOCK < p1) r.dst[d[u]] = acc[u];
    }
  }
}
// A reduction item: wait (bounded) until every evaluation tile of its member has finished, then
// run it.  The wait ends after spin_limit polls; the status word then records bit 2 and the item
// runs on whatever is there, so the kernel always finishes.
static __device__ void exa_step_task(const ExaStep& st, const ExaTask& tk, int* status) {
  const ExaRed& r = st.r[tk.kind - 1];
  if (r.how < 0) return;
  if (threadIdx.x == 0) {
    const int need = __ldg(st.need + tk.member);
    const int* cnt = st.ctr + 1 + tk.member;
    int v = 0, polls = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
      if (v >= need) break;
      if (++polls > st.spin_limit) { atomicOr(status, 2); break; }
      __nanosleep(200);
    }
    __threadfence();
  }
  __syncthreads();
  if (r.how == 0) exa_red_perm(r, tk.p0, tk.p1);
  else exa_red_seg(r, tk.p0, tk.p1);
}
)";

}  // namespace

std::string generate_source(const std::vector<Pattern> &pats, const std::vector<Group> &groups,
                            const CodegenOptions &opt_in, std::string *err, int *dsmem) {
    CodegenOptions opt = opt_in;
    if (opt.lanes > 1) opt.prefetch = 0;  // one or the other
    if (opt.fused_step) {  // the fused step kernels take plain tiles
        opt.stage = 0;
        opt.prefetch = 0;
        opt.lanes = 1;
    }
    if (opt.stage) {  // staging excludes L2 prefetch, warp sets and the bounds-checked indices
        opt.prefetch = 0;
        opt.lanes = 1;
        if (opt.bounds_check) opt.stage = 0;
    }
    if (dsmem)
        for (int m = 0; m < M_COUNT; m++) dsmem[m] = 0;
    std::ostringstream src;
    const bool mixed = opt.precision == EXA_MIXED_FP32;
    src << "// generated by exa_lower.cpp (" << (mixed ? "mixed FP32/FP64" : "FP64") << ")\n";
    src << kDeviceStructs << "\n";
    src << "#define EXA_BLOCK " << opt.block << "\n";
    src << "#define EXA_PF_DEPTH " << opt.prefetch << "\n";
    src << "#define EXA_LANES " << opt.lanes << "\n";
    if (opt.min_blocks > 0) src << "#define EXA_BOUNDS __launch_bounds__(EXA_BLOCK, " << opt.min_blocks << ")\n";
    else src << "#define EXA_BOUNDS __launch_bounds__(EXA_BLOCK)\n";
    if (mixed) src << kMixedHelpers;
    src << kExactHelpers;
    src << kFp64Helpers;
    if (opt.fused_step) src << kStepHelpers;
    if (opt.stage)
        src << "// cp.async of one 8- or 4-byte input into a shared-memory slot (both addresses aligned to\n"
               "// the size: data columns, x and y are arrays of that element size)\n"
               "static __device__ __forceinline__ void exa_cp_async8(const unsigned d, const void* s) {\n"
               "  asm volatile(\"cp.async.ca.shared.global [%0], [%1], 8;\" :: \"r\"(d), \"l\"(s) : \"memory\");\n"
               "}\n"
               "static __device__ __forceinline__ void exa_cp_async4(const unsigned d, const void* s) {\n"
               "  asm volatile(\"cp.async.ca.shared.global [%0], [%1], 4;\" :: \"r\"(d), \"l\"(s) : \"memory\");\n"
               "}\n"
               "extern __shared__ __align__(16) unsigned char exa_dsm[];\n";
    // one shared expression graph per group
    std::vector<Graph> graphs(groups.size());
    std::vector<std::vector<PatternGraph>> pgs(groups.size());
    for (size_t gi = 0; gi < groups.size(); gi++) {
        const Group &grp = groups[gi];
        pgs[gi].resize(grp.pats.size());
        for (size_t pos = 0; pos < grp.pats.size(); pos++) {
            InputMap im{&grp.sym[pos], &grp.field[pos], (int)pos};
            build_graph(pats[grp.pats[pos]], im, graphs[gi], pgs[gi][pos], mixed);
            if (!pgs[gi][pos].err.empty()) {
                *err = pgs[gi][pos].err;
                return "";
            }
        }
    }
    for (int m = 0; m < M_COUNT; m++) {
        std::vector<int> gl;
        std::map<int, int> nsets;  // group -> warp sets (> 1 only when split)
        int S8 = 0, S4 = 0;        // staged slots per thread (largest over the kernel's groups)
        std::vector<int> gst;      // groups with a stage function
        int smax = 1;  // widest slot block staged per warp for the coalesced output writes (ws)
        for (const Pattern &p : pats)
            if (pattern_in_mode(p, (Mode)m)) smax = std::max(smax, std::max(p.nj(), p.nh()));
        if (mode_hess_comp(m))
            for (const Group &gr : groups) smax = std::max(smax, (int)gr.hc.size());
        // staged input slots: two buffers within 160 KB of shared memory per CTA beside ws
        const int st_budget = opt.stage ? std::max(0, (160 * 1024 - opt.block * smax * 8) / (2 * opt.block)) & ~7 : 0;
        for (size_t gi = 0; gi < groups.size(); gi++) {
            bool any = false;
            for (int pid : groups[gi].pats) any = any || pattern_in_mode(pats[pid], (Mode)m);
            if (!any) continue;
            gl.push_back((int)gi);
            Emitter e(pats, groups[gi], graphs[gi], pgs[gi], opt);
            e.st_budget = st_budget;
            const std::vector<std::vector<int>> sets = group_sets(pats, groups[gi], (Mode)m, opt.lanes);
            if (sets.size() == 1) {
                src << e.function((int)gi, (Mode)m, sets[0]);
                src << e.pf_text;
                if (!e.st_text.empty()) {
                    src << e.st_text;
                    gst.push_back((int)gi);
                    S8 = std::max(S8, e.n_st8);
                    S4 = std::max(S4, e.n_st4);
                }
            } else {
                nsets[(int)gi] = (int)sets.size();
                for (size_t si = 0; si < sets.size(); si++)
                    src << e.function((int)gi, (Mode)m, sets[si], "_s" + std::to_string(si));
            }
        }
        const bool objred = (m == M_OBJ || mode_all(m) || m == M_FIRST);
        const bool stk = opt.stage && m != M_STRUCT && !gst.empty();  // staged tile loop
        if (stk) {
            // the staged inputs of tile t, instance clamped like the tile loop's, into the slot
            // columns at shared addresses d8 / d4
            src << "static __device__ __forceinline__ void exa_st_" << kModeName[m]
                << "(const ExaTile* __restrict__ tiles, const ExaPM* __restrict__ pms, const long long t,"
                   " const double* __restrict__ x, const double* __restrict__ y, const unsigned d8, const unsigned d4) {\n"
                   "  const ExaTile tl = tiles[t];\n"
                   "  const ExaPM& pm = pms[tl.pm];\n"
                   "  const int k0 = tl.begin + (int)threadIdx.x;\n"
                   "  const int k = k0 < pm.n_inst ? k0 : (int)pm.n_inst - 1;\n"
                   "  switch (pm.grp) {\n";
            for (int gi : gst)
                src << "    case " << gi << ": grp" << gi << "_" << kModeName[m] << "_st(pm, k, x, y, d8, d4); break;\n";
            src << "    default: break;\n  }\n}\n";
            if (dsmem) dsmem[m] = 2 * opt.block * (8 * S8 + 4 * S4);
        }
        // Tile loop: with gridDim.x == ntiles every CTA takes one tile; a smaller (persistent) grid
        // strides over the tile list.  The trip count is uniform over the CTA.
        src << "extern \"C\" __global__ void EXA_BOUNDS exa_" << kModeName[m]
            << "(const ExaTile* __restrict__ tiles, const int ntiles, const ExaPM* __restrict__ pms,"
               " const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ th,"
               " const double sigma, const ExaOut o, const ExaStructOut so, const int pfd) {\n";
        if (objred) src << "  __shared__ double red[EXA_BLOCK / 32];\n";
        if (m != M_STRUCT)
            src << "  __shared__ double stage[EXA_BLOCK * " << smax << "];\n"
                   "  double* __restrict__ ws = stage + (threadIdx.x & ~31u) * " << smax << ";\n";
        else
            src << "  double* ws = nullptr;\n";
        src << "  double objv = 0.0;\n";
        if (stk) {
            // Two buffers of per-thread slot columns: while tile t computes from one, the CTA's next
            // tile is copied into the other (each thread copies and later reads only its own
            // slots, so the per-thread cp.async group wait is the only synchronisation).
            src << "  double* const sd8 = (double*)exa_dsm;                              // [2][" << S8 << "][EXA_BLOCK]\n"
                   "  int* const sd4 = (int*)(exa_dsm + 2 * " << S8 << " * EXA_BLOCK * 8);  // [2][" << S4 << "][EXA_BLOCK]\n"
                   "  const unsigned sa8 = (unsigned)__cvta_generic_to_shared(sd8 + threadIdx.x);\n"
                   "  const unsigned sa4 = (unsigned)__cvta_generic_to_shared(sd4 + threadIdx.x);\n"
                   "  int sbuf = 0;\n"
                   "  if ((int)blockIdx.x < ntiles) exa_st_" << kModeName[m] << "(tiles, pms, blockIdx.x, x, y, sa8, sa4);\n"
                   "  asm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n";
        }
        src << "  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {\n";
        if (stk) {
            src << "  {\n"
                   "    const long long tn = (long long)t + gridDim.x;\n"
                   "    if (tn < ntiles) exa_st_" << kModeName[m] << "(tiles, pms, tn, x, y, sa8 + (unsigned)(sbuf ^ 1) * (" << S8
                << "u * EXA_BLOCK * 8u), sa4 + (unsigned)(sbuf ^ 1) * (" << S4 << "u * EXA_BLOCK * 4u));\n"
                   "    asm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n"
                   "    asm volatile(\"cp.async.wait_group 1;\" ::: \"memory\");\n"
                   "  }\n"
                   "  const double* __restrict__ s8 = sd8 + sbuf * (" << S8 << " * EXA_BLOCK) + threadIdx.x;\n"
                   "  const int* __restrict__ s4 = sd4 + sbuf * (" << S4 << " * EXA_BLOCK) + threadIdx.x;\n";
        }
        if (opt.prefetch >= 1 && m != M_STRUCT) {  // data columns of the tile 2 x pfd ahead: warp 0
            src << "  if (threadIdx.x < 32 && pfd > 0) {\n"
                   "    const long long tp = (long long)t + 2LL * pfd;\n"
                   "    if (tp < ntiles) {\n"
                   "      const ExaTile tn = tiles[tp];\n"
                   "      const ExaPM& pn = pms[tn.pm];\n"
                   "      switch (pn.grp) {\n";
            for (int gi : gl) src << "        case " << gi << ": grp" << gi << "_" << kModeName[m] << "_pf(pn, tn.begin); break;\n";
            src << "        default: break;\n      }\n    }\n  }\n";
        }
        if (opt.prefetch >= 2 && m != M_STRUCT) {  // x and y lines of the tile pfd ahead: every thread
            src << "  if (pfd > 0) {\n"
                   "    const long long tq = (long long)t + pfd;\n"
                   "    if (tq < ntiles) {\n"
                   "      const ExaTile tn = tiles[tq];\n"
                   "      const ExaPM& pn = pms[tn.pm];\n"
                   "      const int kq = tn.begin + (int)threadIdx.x;\n"
                   "      if (kq < pn.n_inst) switch (pn.grp) {\n";
            for (int gi : gl) src << "        case " << gi << ": grp" << gi << "_" << kModeName[m] << "_pfx(pn, kq, x, y); break;\n";
            src << "        default: break;\n      }\n    }\n  }\n";
        }
        src << "  const ExaTile tl = tiles[t];\n"
               "  const ExaPM& pm = pms[tl.pm];\n";
        if (nsets.empty()) {
            src << "  const int k0 = tl.begin + (int)threadIdx.x;\n";
        } else {
            // split groups: warp set `ws_set` of EXA_BLOCK / nset threads takes the tile's instances
            // for its subset of the group's patterns (sets are whole warps: EXA_BLOCK / 2 is a
            // multiple of 32)
            src << "  int nset = 1;\n  switch (pm.grp) {\n";
            for (auto &kv : nsets) src << "    case " << kv.first << ": nset = " << kv.second << "; break;\n";
            src << "    default: break;\n  }\n"
                   "  const int per = EXA_BLOCK / nset;\n"
                   "  const int ws_set = (int)threadIdx.x / per;\n"
                   "  const int k0 = tl.begin + (int)threadIdx.x - ws_set * per;\n";
        }
        src << "  const bool act = k0 < pm.n_inst;\n"
               "  const int k = act ? k0 : (int)pm.n_inst - 1;\n"
               "  if (__any_sync(0xffffffffu, act)) {\n"
               "    switch (pm.grp) {\n";
        for (int gi : gl) {
            auto it = nsets.find(gi);
            if (it == nsets.end()) {
                src << "      case " << gi << ": grp" << gi << "_" << kModeName[m] << "(pm, k, act, x, y, th, sigma, o, so, objv, ws"
                    << (opt.stage && m != M_STRUCT ? (stk ? ", s8, s4" : ", nullptr, nullptr") : "") << "); break;\n";
            } else {
                src << "      case " << gi << ":\n";
                for (int si = 0; si < it->second; si++)
                    src << "        " << (si ? "else " : "") << "if (ws_set == " << si << ") grp" << gi << "_" << kModeName[m]
                        << "_s" << si << "(pm, k, act, x, y, th, sigma, o, so, objv, ws);\n";
                src << "        break;\n";
            }
        }
        src << "      default: break;\n    }\n  }\n";
        if (stk) src << "  sbuf ^= 1;\n";
        src << "  }\n";
        if (stk) src << "  asm volatile(\"cp.async.wait_group 0;\" ::: \"memory\");  // nothing in flight at exit\n";
        if (objred) {
            // Every thread sums the objective terms of all its instances over the CTA's tiles (in tile
            // order); the CTA reduces once, after its last tile, and writes one partial sum: the
            // partials of a launch are obj_part[0 .. gridDim.x), in a fixed order for a fixed grid.
            // (a warp whose sums are all zero, e.g. one that met no objective instance, skips the
            // shuffle tree: the test is on the bits, on the integer pipe)
            src << "  if (__any_sync(0xffffffffu, (__double_as_longlong(objv) << 1) != 0))\n"
                   "    for (int off = 16; off > 0; off >>= 1) objv += __shfl_xor_sync(0xffffffffu, objv, off);\n"
                   "  else\n"
                   "    objv = 0.0;\n"
                   "  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = objv;\n"
                   "  __syncthreads();\n"
                   "  if (threadIdx.x == 0) {\n"
                   "    double s = 0.0;\n"
                   "    for (int i = 0; i < EXA_BLOCK / 32; i++) s += red[i];\n"
                   "    o.obj_part[blockIdx.x] = s;\n"
                   "  }\n";
        }
        src << "}\n";
        if (opt.fused_step && (m == M_ALL || m == M_ALL_B)) {
            // The fused step: every CTA takes items from one queue until it is empty; an evaluation
            // tile is this kernel kind's tile, after which the CTA counts it for its member; a
            // reduction item waits for its member's tiles (exa_step_task).  Items are queued so
            // that a member's reductions come well after its tiles, and a tile never waits, so the
            // kernel finishes whatever the number of resident CTAs.
            src << "extern \"C\" __global__ void EXA_BOUNDS exa_step" << (m == M_ALL_B ? "_b" : "")
                << "(const ExaTile* __restrict__ tiles, const int ntiles, const ExaPM* __restrict__ pms,"
                   " const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ th,"
                   " const double sigma, const ExaOut o, const ExaStructOut so, const int pfd, const ExaStep st) {\n"
                   "  __shared__ double red[EXA_BLOCK / 32];\n"
                   "  __shared__ double stage[EXA_BLOCK * " << smax << "];\n"
                   "  __shared__ int s_item;\n"
                   "  double* __restrict__ ws = stage + (threadIdx.x & ~31u) * " << smax << ";\n"
                   "  double objv = 0.0;\n"
                   "  for (;;) {\n"
                   "    if (threadIdx.x == 0) s_item = atomicAdd(st.ctr, 1);\n"
                   "    __syncthreads();\n"
                   "    const int it = s_item;\n"
                   "    __syncthreads();\n"
                   "    if (it >= st.nitems) break;\n"
                   "    const ExaTask tk = st.items[it];\n"
                   "    if (tk.kind != 0) { exa_step_task(st, tk, o.status); continue; }\n"
                   "    const ExaTile tl = tiles[tk.p0];\n"
                   "    const ExaPM& pm = pms[tl.pm];\n"
                   "    const int k0 = tl.begin + (int)threadIdx.x;\n"
                   "    const bool act = k0 < pm.n_inst;\n"
                   "    const int k = act ? k0 : (int)pm.n_inst - 1;\n"
                   "    if (__any_sync(0xffffffffu, act)) {\n"
                   "      switch (pm.grp) {\n";
            for (int gi : gl)
                src << "        case " << gi << ": grp" << gi << "_" << kModeName[m]
                    << "(pm, k, act, x, y, th, sigma, o, so, objv, ws); break;\n";
            src << "        default: break;\n      }\n    }\n"
                   "    __syncthreads();\n"
                   "    if (threadIdx.x == 0) { __threadfence(); atomicAdd(st.ctr + 1 + tk.member, 1); }\n"
                   "  }\n"
                   "  if (__any_sync(0xffffffffu, (__double_as_longlong(objv) << 1) != 0))\n"
                   "    for (int off = 16; off > 0; off >>= 1) objv += __shfl_xor_sync(0xffffffffu, objv, off);\n"
                   "  else\n"
                   "    objv = 0.0;\n"
                   "  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = objv;\n"
                   "  __syncthreads();\n"
                   "  if (threadIdx.x == 0) {\n"
                   "    double s = 0.0;\n"
                   "    for (int i = 0; i < EXA_BLOCK / 32; i++) s += red[i];\n"
                   "    o.obj_part[blockIdx.x] = s;\n"
                   "  }\n"
                   "}\n";
        }
    }
    return src.str();
}

}  // namespace exa
