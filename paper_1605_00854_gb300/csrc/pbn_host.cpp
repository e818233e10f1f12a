/*
 * pbn_host.cpp -- host-side preparation of the structure-based PBN simulation.
 *
 *   pbn_load      network text -> model G(X, F) with probabilities C_i      (Sec. 2.1)
 *   pbn_reduce    leaf-node reduction                             (Sec. 3.1, Definition 1)
 *   pbn_group     node grouping and merged predictor functions    (Sec. 3.3, Eq. 2, Alg. 3-4)
 *                 and the device image of Algorithm 5's Preparation
 *   pbn_estimate  two-state Markov chain estimate                  (Sec. 4.2)
 */
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include "pbn_internal.h"

namespace {
thread_local std::string g_detail;
}

namespace pbn {
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_detail = buf;
    return code;
}

/* Node i is perturbed iff its 32-bit draw u < P = floor(p * 2^32); p * 2^32 is exact. */
uint64_t pert_threshold(double p) { return (uint64_t)std::floor(p * 4294967296.0); }

int meta_rows(const pbn_plan* plan, const uint32_t* ids, const uint8_t* vals, uint32_t n_meta, uint32_t max_rows,
              const char* who, MetaRows* out) {
    *out = MetaRows{};
    if (max_rows > 64) max_rows = 64;
    for (uint32_t m = 0; m < n_meta; ++m) {
        const uint32_t id = ids[m];
        if (id >= plan->hdr.n || plan->pos[id] == UINT32_MAX)
            return fail(PBN_EINVAL, "%s: meta node %u is not a retained node", who, id);
        const uint32_t row = plan->pos[id] >> 5, bit = plan->pos[id] & 31u;
        const uint32_t val = vals ? (vals[m] ? 1u : 0u) : 1u;
        uint32_t k = 0;
        while (k < out->n_rows && out->row[k] != row) ++k;
        if (k == out->n_rows) {
            if (k == max_rows) return fail(PBN_EINVAL, "%s: meta nodes span more than %u state words", who, max_rows);
            out->row[k] = row;
            out->mask[k] = 0;
            out->val[k] = 0;
            out->n_rows++;
        }
        if (((out->mask[k] >> bit) & 1u) && ((out->val[k] >> bit) & 1u) != val)
            return fail(PBN_EINVAL, "%s: contradictory values for meta node %u", who, id);
        out->mask[k] |= 1u << bit;
        out->val[k] |= val << bit;
    }
    return PBN_OK;
}
}  // namespace pbn

using pbn::fail;

extern "C" const char* pbn_last_error_detail(void) { return g_detail.c_str(); }

extern "C" const char* pbn_strerror(int s) {
    switch (s) {
        case PBN_OK: return "ok";
        case PBN_EINVAL: return "invalid argument";
        case PBN_EPARSE: return "malformed network text";
        case PBN_ENOMEM: return "out of host memory";
        case PBN_ECUDA: return "CUDA error";
        case PBN_ETOOBIG: return "plan exceeds device limits";
        case PBN_ETIMEOUT: return "bounded device wait timed out";
        case PBN_EDEVICE: return "kernel reported an error";
        default: return "unknown status";
    }
}

extern "C" const char* pbn_version(void) { return "pbn-gb300 1.0 (sm_103a)"; }

/* ------------------------------------------------------------------------- */
/* Parsing                                                                    */
/* ------------------------------------------------------------------------- */
namespace {

bool parse_u64(const std::string& t, uint64_t* v) {
    if (t.empty()) return false;
    char* end = nullptr;
    errno = 0;
    unsigned long long x = std::strtoull(t.c_str(), &end, 10);
    if (errno || *end || t[0] == '-') return false;
    *v = x;
    return true;
}

bool parse_f64(const std::string& t, double* v) {
    if (t.empty()) return false;
    char* end = nullptr;
    double x = std::strtod(t.c_str(), &end);
    if (*end) return false;
    *v = x;
    return true;
}

int nibble(char ch) {
    if (ch >= '0' && ch <= '9') return ch - '0';
    if (ch >= 'a' && ch <= 'f') return 10 + ch - 'a';
    if (ch >= 'A' && ch <= 'F') return 10 + ch - 'A';
    return -1;
}

/* Split one line into whitespace-separated tokens, dropping a '#' comment. */
void tokenize(const char* b, const char* e, std::vector<std::string>* out) {
    out->clear();
    const char* hash = static_cast<const char*>(memchr(b, '#', (size_t)(e - b)));
    if (hash) e = hash;
    const char* p = b;
    while (p < e) {
        while (p < e && (*p == ' ' || *p == '\t' || *p == '\r')) ++p;
        const char* q = p;
        while (q < e && *q != ' ' && *q != '\t' && *q != '\r') ++q;
        if (q > p) out->emplace_back(p, q);
        p = q;
    }
}

int finish_net(pbn_net* g, int code, pbn_net** out);

int load_impl(const char* text, size_t len, pbn_net** out) {
    pbn_net* g = new pbn_net();
    std::vector<std::string> tok;
    const char* p = text;
    const char* end = text + len;
    bool have_header = false;
    size_t lineno = 0;
    while (p < end) {
        const char* nl = static_cast<const char*>(memchr(p, '\n', (size_t)(end - p)));
        const char* le = nl ? nl : end;
        ++lineno;
        tokenize(p, le, &tok);
        p = nl ? nl + 1 : end;
        if (tok.empty()) continue;
        if (tok[0] == "pbn") {
            uint64_t n;
            double pr;
            if (have_header || tok.size() != 3 || !parse_u64(tok[1], &n) || !parse_f64(tok[2], &pr) ||
                n < 1 || n > (1u << 24) || !(pr >= 0.0 && pr < 1.0)) {
                delete g;
                return fail(PBN_EPARSE, "line %zu: bad 'pbn <n> <p>' header", lineno);
            }
            have_header = true;
            g->n = (uint32_t)n;
            g->p = pr;
            g->node.assign(n, {});
        } else if (tok[0] == "f") {
            uint64_t i, k;
            double c;
            if (!have_header || tok.size() < 5 || !parse_u64(tok[1], &i) || !parse_f64(tok[2], &c) ||
                !parse_u64(tok[3], &k) || i >= g->n || k > 24 || !(c >= 0.0 && c <= 1.0) ||
                tok.size() != 5 + k) {
                delete g;
                return fail(PBN_EPARSE, "line %zu: bad function record", lineno);
            }
            pbn_fun f;
            f.c = c;
            for (uint64_t b = 0; b < k; ++b) {
                uint64_t a;
                if (!parse_u64(tok[4 + b], &a) || a >= g->n ||
                    std::find(f.par.begin(), f.par.end(), (uint32_t)a) != f.par.end()) {
                    delete g;
                    return fail(PBN_EPARSE, "line %zu: bad or repeated parent", lineno);
                }
                f.par.push_back((uint32_t)a);
            }
            std::string hex = tok[4 + k];
            if (hex.size() > 2 && hex[0] == '0' && (hex[1] == 'x' || hex[1] == 'X')) hex = hex.substr(2);
            const uint64_t nbits = 1ull << k;
            f.tt.assign((nbits + 63) / 64, 0);
            if (hex.empty()) {
                delete g;
                return fail(PBN_EPARSE, "line %zu: empty truth table", lineno);
            }
            for (size_t d = 0; d < hex.size(); ++d) {
                int v = nibble(hex[hex.size() - 1 - d]);
                if (v < 0) {
                    delete g;
                    return fail(PBN_EPARSE, "line %zu: bad hex digit", lineno);
                }
                for (int b = 0; b < 4; ++b) {
                    if (!((v >> b) & 1)) continue;
                    uint64_t bit = 4 * (uint64_t)d + (uint64_t)b;
                    if (bit >= nbits) {
                        delete g;
                        return fail(PBN_EPARSE, "line %zu: truth table wider than 2^k bits", lineno);
                    }
                    f.tt[bit >> 6] |= 1ull << (bit & 63);
                }
            }
            g->node[i].push_back(std::move(f));
        } else {
            delete g;
            return fail(PBN_EPARSE, "line %zu: unknown record '%s'", lineno, tok[0].c_str());
        }
    }
    if (!have_header) {
        delete g;
        return fail(PBN_EPARSE, "missing 'pbn' header");
    }
    return finish_net(g, PBN_EPARSE, out);
}

/* Per-node requirements shared by both loaders; takes ownership of g. */
int finish_net(pbn_net* g, int code, pbn_net** out) {
    for (uint32_t i = 0; i < g->n; ++i) {
        const auto& fl = g->node[i];
        if (fl.empty() || fl.size() > 16) {
            const size_t nf = fl.size();
            delete g;
            return fail(code, "node %u has %zu functions (need 1..16)", i, nf);
        }
        double s = 0.0;
        for (const auto& f : fl) s += f.c;
        if (std::fabs(s - 1.0) > 1e-9) {
            delete g;
            return fail(code, "selection probabilities of node %u sum to %.17g", i, s);
        }
    }
    g->retained.assign(g->n, 1);
    *out = g;
    return PBN_OK;
}

int load_arrays_impl(const pbn_net_desc* d, pbn_net** out) {
    if (d->n < 1 || d->n > (1u << 24) || !(d->p >= 0.0 && d->p < 1.0))
        return fail(PBN_EINVAL, "pbn_load_arrays: need 1 <= n <= 2^24 and 0 <= p < 1");
    if (d->n_functions && (!d->fun_node || !d->fun_c || !d->fun_k || !d->tt))
        return fail(PBN_EINVAL, "pbn_load_arrays: NULL array");
    std::unique_ptr<pbn_net> g(new pbn_net());
    g->n = d->n;
    g->p = d->p;
    g->node.assign(d->n, {});
    uint64_t po = 0, to = 0;
    for (uint32_t f = 0; f < d->n_functions; ++f) {
        const uint32_t i = d->fun_node[f], k = d->fun_k[f];
        const double c = d->fun_c[f];
        if (i >= d->n || k > 24 || !(c >= 0.0 && c <= 1.0))
            return fail(PBN_EINVAL, "pbn_load_arrays: function %u: bad node, k or c", f);
        if (k && !d->parents) return fail(PBN_EINVAL, "pbn_load_arrays: NULL parents");
        pbn_fun fn;
        fn.c = c;
        for (uint32_t b = 0; b < k; ++b) {
            const uint32_t a = d->parents[po + b];
            if (a >= d->n || std::find(fn.par.begin(), fn.par.end(), a) != fn.par.end())
                return fail(PBN_EINVAL, "pbn_load_arrays: function %u: bad or repeated parent", f);
            fn.par.push_back(a);
        }
        po += k;
        const uint64_t nbits = 1ull << k, nw = (nbits + 63) / 64;
        fn.tt.assign(d->tt + to, d->tt + to + nw);
        to += nw;
        if (nbits < 64 && (fn.tt[0] >> nbits))
            return fail(PBN_EINVAL, "pbn_load_arrays: function %u: truth table wider than 2^k bits", f);
        g->node[i].push_back(std::move(fn));
    }
    return finish_net(g.release(), PBN_EINVAL, out);
}

}  // namespace

extern "C" int pbn_load(const char* text, size_t len, pbn_net** out) {
    if (!text || !out) return fail(PBN_EINVAL, "pbn_load: NULL argument");
    *out = nullptr;
    try {
        return load_impl(text, len, out);
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_load: out of memory");
    }
}

extern "C" int pbn_load_arrays(const pbn_net_desc* desc, pbn_net** out) {
    if (!desc || !out) return fail(PBN_EINVAL, "pbn_load_arrays: NULL argument");
    *out = nullptr;
    try {
        return load_arrays_impl(desc, out);
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_load_arrays: out of memory");
    }
}

extern "C" void pbn_net_free(pbn_net* net) { delete net; }

extern "C" int pbn_net_info_get(const pbn_net* g, pbn_net_info* out) {
    if (!g || !out) return fail(PBN_EINVAL, "pbn_net_info_get: NULL argument");
    memset(out, 0, sizeof(*out));
    out->n = g->n;
    out->p = g->p;
    out->P = pbn::pert_threshold(g->p);
    uint64_t sum_par = 0;
    for (uint32_t i = 0; i < g->n; ++i) {
        out->n_retained += g->retained[i];
        out->n_functions += (uint32_t)g->node[i].size();
        out->n_multi += g->node[i].size() >= 2;
        for (const auto& f : g->node[i]) sum_par += f.par.size();
    }
    out->density = (double)sum_par / (double)g->n;
    return PBN_OK;
}

/* ------------------------------------------------------------------------- */
/* Leaf-node reduction, Definition 1 (Sec. 3.1).  Peeling: a node not of       */
/* interest whose count of not-yet-removed children (self-edges excluded)     */
/* reaches zero is a leaf; removing it decrements its parents' counts.        */
/* ------------------------------------------------------------------------- */
extern "C" int pbn_reduce(const pbn_net* net, const uint32_t* interest, uint32_t n_interest,
                          pbn_net** reduced, uint32_t* retained_ids, uint32_t* n_retained) {
    return pbn_reduce_rule(net, interest, n_interest, PBN_REDUCE_LEAVES, reduced, retained_ids, n_retained);
}

extern "C" int pbn_reduce_rule(const pbn_net* net, const uint32_t* interest, uint32_t n_interest, uint32_t rule,
                               pbn_net** reduced, uint32_t* retained_ids, uint32_t* n_retained) {
    if (!net || !reduced || (n_interest && !interest)) return fail(PBN_EINVAL, "pbn_reduce: NULL argument");
    if (rule != PBN_REDUCE_LEAVES && rule != PBN_REDUCE_REACH) return fail(PBN_EINVAL, "pbn_reduce: unknown rule %u", rule);
    *reduced = nullptr;
    try {
        const uint32_t n = net->n;
        std::vector<uint8_t> intr(n, 0);
        for (uint32_t m = 0; m < n_interest; ++m) {
            if (interest[m] >= n) return fail(PBN_EINVAL, "pbn_reduce: node of interest %u >= n", interest[m]);
            intr[interest[m]] = 1;
        }
        std::vector<std::vector<uint32_t>> parents(n);  /* distinct parents of u, u excluded */
        std::vector<uint32_t> live_children(n, 0);
        for (uint32_t u = 0; u < n; ++u) {
            auto& pu = parents[u];
            for (const auto& f : net->node[u])
                for (uint32_t a : f.par)
                    if (a != u) pu.push_back(a);
            std::sort(pu.begin(), pu.end());
            pu.erase(std::unique(pu.begin(), pu.end()), pu.end());
            for (uint32_t a : pu) live_children[a]++;
        }
        std::vector<uint8_t> leaf(n, 0);
        std::vector<uint32_t> stack;
        if (rule == PBN_REDUCE_LEAVES) {
            for (uint32_t v = 0; v < n; ++v)
                if (!intr[v] && live_children[v] == 0) { leaf[v] = 1; stack.push_back(v); }
            while (!stack.empty()) {
                uint32_t v = stack.back();
                stack.pop_back();
                for (uint32_t a : parents[v]) {
                    if (--live_children[a] == 0 && !intr[a] && !leaf[a]) {
                        leaf[a] = 1;
                        stack.push_back(a);
                    }
                }
            }
        } else {
            /* search backwards from the nodes of interest along child -> parent */
            std::vector<uint8_t> reach(n, 0);
            for (uint32_t v = 0; v < n; ++v)
                if (intr[v]) { reach[v] = 1; stack.push_back(v); }
            while (!stack.empty()) {
                uint32_t v = stack.back();
                stack.pop_back();
                for (uint32_t a : parents[v])
                    if (!reach[a]) { reach[a] = 1; stack.push_back(a); }
            }
            for (uint32_t v = 0; v < n; ++v) leaf[v] = !reach[v];
        }
        pbn_net* r = new pbn_net(*net);
        uint32_t cnt = 0;
        for (uint32_t v = 0; v < n; ++v) {
            r->retained[v] = (uint8_t)(net->retained[v] && !leaf[v]);
            if (r->retained[v]) {
                if (retained_ids) retained_ids[cnt] = v;
                ++cnt;
            }
        }
        r->interest.assign(interest, interest + n_interest);
        if (n_retained) *n_retained = cnt;
        *reduced = r;
        return PBN_OK;
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_reduce: out of memory");
    }
}

/* ------------------------------------------------------------------------- */
/* Grouping (Sec. 3.3)                                                        */
/* ------------------------------------------------------------------------- */
namespace {

struct Item {
    uint32_t id;
    uint32_t ell;                  /* l(v) = omega(mu) */
    std::vector<uint32_t> inputs;  /* sorted distinct parents over all functions */
};

struct Grp {
    std::vector<uint32_t> nodes;   /* in output bit order (right to left) */
    std::vector<uint32_t> inputs;  /* sorted distinct inputs */
    uint64_t weight = 0;           /* prod l(v) over members; 0 when empty */
    bool multi = false;
};

uint64_t sat_mul(uint64_t a, uint64_t b) {
    if (a == 0 || b == 0) return 0;
    if (a > (UINT64_C(1) << 62) / b) return UINT64_C(1) << 62;
    return a * b;
}

size_t union_size(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    size_t i = 0, j = 0, u = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) { ++i; ++j; }
        else if (a[i] < b[j]) ++i;
        else ++j;
        ++u;
    }
    return u + (a.size() - i) + (b.size() - j);
}

size_t inter_size(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    return a.size() + b.size() - union_size(a, b);
}

void merge_into(std::vector<uint32_t>* a, const std::vector<uint32_t>& b) {
    std::vector<uint32_t> out;
    out.reserve(a->size() + b.size());
    std::set_union(a->begin(), a->end(), b.begin(), b.end(), std::back_inserter(out));
    a->swap(out);
}

uint32_t log2_entry_bits(uint32_t width) {
    uint32_t l = 0;
    while ((1u << l) < width) ++l;
    return l;
}

/* Bits of a merged table: prod l(v) * 2^q entries of 2^ceil(log2 width) bits. */
double table_bits(uint64_t prod_ell, size_t q, size_t width) {
    return (double)prod_ell * std::ldexp(1.0, (int)q) * (double)(1u << log2_entry_bits((uint32_t)width));
}

constexpr double kMaxTableBits = 1073741824.0; /* 2^30 */

struct Caps {
    uint32_t max_inputs, max_width;
};

bool can_join(const Grp& g, const Item& it, const Caps& cp) {
    if (g.nodes.empty()) return true;
    if (g.nodes.size() + 1 > cp.max_width) return false;
    size_t q = union_size(g.inputs, it.inputs);
    if (q > cp.max_inputs) return false;
    return table_bits(sat_mul(g.weight, it.ell), q, g.nodes.size() + 1) <= kMaxTableBits;
}

void join(Grp* g, const Item& it) {
    g->weight = g->nodes.empty() ? it.ell : sat_mul(g->weight, it.ell);
    g->nodes.push_back(it.id);
    merge_into(&g->inputs, it.inputs);
}

/* Algorithm 3 (FindPartitions): items sorted by descending weight (ties: ascending
 * id); each goes to the lightest of the m groups (an empty group weighs 0; ties:
 * lowest index) among those it may join under the GPU caps.  Returns the number of
 * items no group could take. */
size_t find_partitions(const std::vector<Item>& S, size_t m, const Caps& cp, std::vector<Grp>* out) {
    std::vector<Grp> A(m);
    /* groups ordered by (weight, index): the first feasible one in this order is the
     * lightest feasible group with ties to the lowest index */
    std::set<std::pair<uint64_t, size_t>> order;
    for (size_t i = 0; i < m; ++i) order.insert({0, i});
    size_t unplaced = 0;
    for (const Item& it : S) {
        size_t best = SIZE_MAX;
        for (auto o = order.begin(); o != order.end(); ++o) {
            if (can_join(A[o->second], it, cp)) {
                best = o->second;
                order.erase(o);
                break;
            }
        }
        if (best == SIZE_MAX) { ++unplaced; continue; }
        join(&A[best], it);
        order.insert({A[best].weight, best});
    }
    out->swap(A);
    return unplaced;
}

/* Eq. 2: the smallest m^ with m^ * (prod omega)^(1/m^) <= theta (Theorem 2: a lower
 * bound on any feasible m).  Evaluated in logarithms; m^ (prod)^(1/m^) is smallest
 * near m^ = ln(prod), so the scan stops there.  Returns 0 if no m^ satisfies it. */
uint32_t eq2_lower_bound(const std::vector<Item>& S, double theta) {
    double L = 0.0;
    for (const Item& it : S) L += std::log((double)it.ell);
    const double lt = std::log(theta);
    const uint64_t stop = std::max<uint64_t>((uint64_t)S.size(), (uint64_t)std::ceil(L) + 2);
    for (uint64_t m = 1; m <= stop; ++m)
        if (std::log((double)m) + L / (double)m <= lt + 1e-12) return (uint32_t)m;
    return 0;
}

struct PlanParts {
    std::vector<Grp> groups;
    uint32_t m_lower = 0, m_found = 0;
    uint64_t sum_w = 0;
};

/* Algorithm 4 (Partition) for the retained nodes, plus the common-parent greedy for
 * single-function nodes (Sec. 3.3). */
void partition(const pbn_net& g, const pbn_group_params& prm, PlanParts* pp) {
    Caps cp{prm.max_inputs, prm.max_width};
    std::vector<Item> S, S1;
    for (uint32_t v = 0; v < g.n; ++v) {
        if (!g.retained[v]) continue;
        Item it;
        it.id = v;
        it.ell = (uint32_t)g.node[v].size();
        for (const auto& f : g.node[v]) it.inputs.insert(it.inputs.end(), f.par.begin(), f.par.end());
        std::sort(it.inputs.begin(), it.inputs.end());
        it.inputs.erase(std::unique(it.inputs.begin(), it.inputs.end()), it.inputs.end());
        (it.ell >= 2 ? S : S1).push_back(std::move(it));
    }
    if (prm.mode == PBN_PLAN_PLAIN) {
        std::vector<Item> all;
        all.insert(all.end(), S.begin(), S.end());
        all.insert(all.end(), S1.begin(), S1.end());
        std::sort(all.begin(), all.end(), [](const Item& a, const Item& b) { return a.id < b.id; });
        for (const Item& it : all) {
            Grp gr;
            join(&gr, it);
            gr.multi = it.ell >= 2;
            pp->groups.push_back(std::move(gr));
        }
        return;
    }
    /* multi-function nodes: Eq. 2 lower bound, then Algorithm 3 with m grown until
     * the weight sum is within theta (and the caps hold) */
    std::stable_sort(S.begin(), S.end(), [](const Item& a, const Item& b) {
        return a.ell != b.ell ? a.ell > b.ell : a.id < b.id;
    });
    if (!S.empty()) {
        pp->m_lower = eq2_lower_bound(S, prm.theta);
        size_t m = pp->m_lower ? std::min<size_t>(pp->m_lower, S.size()) : S.size();
        std::vector<Grp> A;
        for (;;) {
            size_t unplaced = find_partitions(S, m, cp, &A);
            uint64_t sum = 0;
            for (const Grp& gr : A) sum += gr.weight;
            if ((unplaced == 0 && (double)sum <= prm.theta) || m >= S.size()) {
                pp->sum_w = sum;
                break;
            }
            m = std::min(S.size(), m + std::max<size_t>(1, unplaced));
        }
        pp->m_found = (uint32_t)m;
        for (Grp& gr : A) {
            if (gr.nodes.empty()) continue;
            gr.multi = true;
            pp->groups.push_back(std::move(gr));
        }
    }
    /* single-function nodes: visit by descending number of parents (ties: id); join
     * the feasible group sharing most parents (ties: lowest index), else open one */
    std::stable_sort(S1.begin(), S1.end(), [](const Item& a, const Item& b) {
        return a.inputs.size() != b.inputs.size() ? a.inputs.size() > b.inputs.size() : a.id < b.id;
    });
    std::vector<Grp> A2;
    for (const Item& it : S1) {
        size_t best = SIZE_MAX, best_shared = 0;
        for (size_t i = 0; i < A2.size(); ++i) {
            if (!can_join(A2[i], it, cp)) continue;
            size_t sh = inter_size(A2[i].inputs, it.inputs);
            if (best == SIZE_MAX || sh > best_shared) { best = i; best_shared = sh; }
        }
        if (best == SIZE_MAX) {
            A2.emplace_back();
            best = A2.size() - 1;
        }
        join(&A2[best], it);
    }
    for (Grp& gr : A2) pp->groups.push_back(std::move(gr));
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

/* Thresholds of the geometric perturbation sampler:
 * G[k] = floor(2^64 (1 - (1 - P/2^32)^(k+1))), k = 0..63.  With a = 2^32 - P the
 * power is a^(k+1) / 2^(32(k+1)), so G[k] = 2^64 - ceil(a^(k+1) 2^(64 - 32(k+1)));
 * a^(k+1) is built exactly in 32-bit limbs (at most 2048 bits). */
void geometric_thresholds(uint32_t P, uint64_t G[64]) {
    if (P == 0) {
        for (int k = 0; k < 64; ++k) G[k] = 0;
        return;
    }
    const uint64_t a = (UINT64_C(1) << 32) - P;
    std::vector<uint32_t> pw(1, 1u); /* a^(k+1), least significant limb first */
    for (int k = 0; k < 64; ++k) {
        uint64_t carry = 0;
        for (uint32_t& l : pw) {
            const uint64_t v = (uint64_t)l * a + carry;
            l = (uint32_t)v;
            carry = v >> 32;
        }
        if (carry) pw.push_back((uint32_t)carry);
        uint64_t q;
        if (k == 0) {
            q = a << 32;
        } else {
            /* a^(k+1) / 2^(32 (k - 1)), rounded up: limbs k-1 and k, plus one if any
             * lower limb is nonzero */
            const size_t lo = (size_t)k - 1;
            q = (lo < pw.size() ? pw[lo] : 0u) | ((uint64_t)(lo + 1 < pw.size() ? pw[lo + 1] : 0u) << 32);
            bool rem = false;
            for (size_t i = 0; i < lo && i < pw.size(); ++i) rem = rem || pw[i] != 0;
            q += rem ? 1u : 0u;
        }
        G[k] = (uint64_t)0 - q;
    }
}

/* ---- Algorithm 5's Preparation: the device image, built stage by stage ------------ */

/* The sections of the device image under construction (layout in pbn_image.h). */
struct ImageBuild {
    uint32_t n = 0, W = 0, W32 = 0;
    std::vector<uint32_t> rank;               /* SEL rank of each node with >= 2 functions */
    std::vector<std::vector<size_t>> in_word; /* partition groups of each 32-bit state word */
    std::vector<uint32_t> gword, gshift;      /* word and bit offset of each partition group */
    std::vector<uint32_t> selblk;             /* SEL blocks drawn per step */
    std::vector<uint32_t> words, selslot, thr, inrec, tables;
    std::vector<uint32_t> subs;    /* uint2 per function of a split node: in_chunk | k << 27, tab_off */
    std::vector<uint32_t> gorder;  /* group index | output word << 20, in evaluation order */
    std::vector<uint32_t> wgroups; /* group indices of each output word (words ranges into it) */
    std::vector<pbn_img_group> grec;
    std::vector<pbn_img_multi> mrec;
    uint32_t n_multi_nodes = 0, n_split = 0, n_groups_multi = 0;
    uint64_t total_inputs = 0;

    /* record of SEL slot s = 4 i + l at l * n_sel + i: lanes that take consecutive
     * blocks read consecutive records */
    uint32_t slot_rec(uint32_t slot) const { return 4 * ((slot & 3u) * (uint32_t)selblk.size() + (slot >> 2)); }
    /* SEL slot of node v: 4 x (position of its block in selblk) + rank mod 4 */
    uint32_t sel_slot(uint32_t v) const {
        const uint32_t b = rank[v] >> 2;
        const uint32_t idx = (uint32_t)(std::lower_bound(selblk.begin(), selblk.end(), b) - selblk.begin());
        return 4 * idx + (rank[v] & 3);
    }
};

/* Input record of input b at state position ps: the row's byte offset above 5
 * rotation bits; the rotation brings the bit to position b mod 4 of its 4-input chunk. */
uint32_t input_record(uint32_t ps, size_t b) { return ((ps >> 5) << 7) | (((ps & 31) - (uint32_t)(b & 3)) & 31); }

/* Groups packed into 32-bit state words, first fit by decreasing width; the word
 * count is even (the state is stored as uint64 words). */
void pack_words(const PlanParts& pp, ImageBuild* B) {
    std::vector<size_t> order(pp.groups.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return pp.groups[a].nodes.size() > pp.groups[b].nodes.size();
    });
    std::vector<uint32_t> fill; /* used bits per word */
    B->gword.assign(pp.groups.size(), 0u);
    B->gshift.assign(pp.groups.size(), 0u);
    for (size_t gi : order) {
        const uint32_t w = (uint32_t)pp.groups[gi].nodes.size();
        size_t k = 0;
        while (k < fill.size() && fill[k] + w > 32) ++k;
        if (k == fill.size()) {
            fill.push_back(0);
            B->in_word.emplace_back();
        }
        B->gword[gi] = (uint32_t)k;
        B->gshift[gi] = fill[k];
        fill[k] += w;
        B->in_word[k].push_back(gi);
    }
    const uint32_t W32 = fill.empty() ? 2u : (uint32_t)fill.size();
    B->W32 = (W32 + 1) & ~1u;
    B->in_word.resize(B->W32);
}

/* State position (32 x word + bit) of every retained node, and its group in the
 * word-by-word evaluation order. */
void place_nodes(const PlanParts& pp, const ImageBuild& B, pbn_plan* plan) {
    plan->pos.assign(B.n, UINT32_MAX);
    plan->group_of.assign(B.n, UINT32_MAX);
    uint32_t e = 0;
    for (uint32_t k = 0; k < B.W32; ++k)
        for (size_t gi : B.in_word[k]) {
            const Grp& gr = pp.groups[gi];
            for (size_t i = 0; i < gr.nodes.size(); ++i) {
                plan->pos[gr.nodes[i]] = 32 * B.gword[gi] + B.gshift[gi] + (uint32_t)i;
                plan->group_of[gr.nodes[i]] = e;
            }
            ++e;
        }
}

/* SEL ranks over every node with >= 2 functions (leaves included), and the SEL
 * Philox blocks that hold the ranks of retained multi-function nodes. */
void sel_blocks(const pbn_net& g, ImageBuild* B) {
    B->rank.assign(B->n, UINT32_MAX);
    uint32_t r = 0;
    for (uint32_t v = 0; v < B->n; ++v)
        if (g.node[v].size() >= 2) B->rank[v] = r++;
    for (uint32_t v = 0; v < B->n; ++v)
        if (g.retained[v] && B->rank[v] != UINT32_MAX) B->selblk.push_back(B->rank[v] >> 2);
    std::sort(B->selblk.begin(), B->selblk.end());
    B->selblk.erase(std::unique(B->selblk.begin(), B->selblk.end()), B->selblk.end());
    B->selslot.assign(16 * B->selblk.size(), 0u);
}

/* Multi record of node v (its SEL slot and mixed-radix weight) and the slot's integer
 * thresholds T_j = floor(C_j 2^32) with C_j summed left to right (a threshold of 2^32
 * never fires and is left out), the first two inline in the slot record. */
void add_choice(const pbn_net& g, uint32_t v, uint32_t radix, ImageBuild* B) {
    const auto& fl = g.node[v];
    const uint32_t first = (uint32_t)B->thr.size();
    double C = 0.0;
    uint32_t n_thr = 0;
    for (size_t j = 1; j < fl.size(); ++j) {
        C = C + fl[j - 1].c;
        const double t = std::floor(C * 4294967296.0);
        if (t >= 4294967296.0) break;
        B->thr.push_back((uint32_t)t);
        n_thr++;
    }
    const uint32_t slot = B->sel_slot(v);
    uint32_t* ss = &B->selslot[B->slot_rec(slot)];
    ss[0] = n_thr >= 1 ? B->thr[first] : 0u;
    ss[1] = n_thr >= 2 ? B->thr[first + 1] : 0u;
    ss[2] = n_thr;
    ss[3] = first;
    pbn_img_multi M{};
    M.ch_off = slot;
    M.radix = radix;
    B->mrec.push_back(M);
}

/* A split node: a lone multi-function node whose input union exceeds the merge cap
 * keeps one table of 2^k one-bit entries per predictor function, over that
 * function's own k inputs, instead of l x 2^q entries over the union; its choice
 * selects the function to evaluate. */
int add_split_group(const pbn_net& g, const pbn_plan& plan, uint32_t v, uint32_t shift, ImageBuild* B) {
    const auto& fl = g.node[v];
    pbn_img_group G{};
    G.mul_first = (uint32_t)B->mrec.size();
    add_choice(g, v, 1u, B);
    G.tab_off = (uint32_t)(B->subs.size() / 2); /* first sub-function */
    G.in_chunk = 0;
    G.q = (uint8_t)fl.size();
    G.l2w = PBN_IMG_SPLIT;
    G.n_mul = 1;
    G.shift = (uint8_t)shift;
    for (const pbn_fun& f : fl) {
        const uint32_t chunk = (uint32_t)(B->inrec.size() / 4);
        for (size_t b = 0; b < f.par.size(); ++b) {
            const uint32_t ps = plan.pos[f.par[b]];
            if (ps == UINT32_MAX) return fail(PBN_EINVAL, "input %u of a retained node was removed", f.par[b]);
            B->inrec.push_back(input_record(ps, b));
        }
        while (B->inrec.size() % 4) B->inrec.push_back(B->W32 << 7); /* the always-zero row */
        const uint32_t k = (uint32_t)f.par.size();
        const uint32_t to = (uint32_t)B->tables.size();
        if (chunk >= (1u << 27)) return fail(PBN_ETOOBIG, "input records beyond 2^27 chunks");
        B->subs.push_back(chunk | (k << 27));
        B->subs.push_back(to);
        const uint64_t nb = 1ull << k;
        B->tables.resize(B->tables.size() + (size_t)((nb + 31) / 32), 0);
        uint32_t* tab = B->tables.data() + to;
        for (uint64_t x = 0; x < nb; ++x) tab[x >> 5] |= (uint32_t)f.bit(x) << (x & 31);
    }
    /* one function's inputs are read per step: count their mean */
    uint64_t ksum = 0;
    for (const pbn_fun& f : fl) ksum += f.par.size();
    B->total_inputs += (ksum + fl.size() - 1) / fl.size();
    B->grec.push_back(G);
    B->n_split++;
    return PBN_OK;
}

/* A merged group (Sec. 3.3): one table over the union of its members' q inputs
 * (`ins`, sorted by state position); entry (c << q) | x, with c the mixed-radix
 * combined choice of the multi-function members (in group bit order) and x the packed
 * input pattern, holds in bit i member i's selected function evaluated on x. */
int add_merged_group(const pbn_net& g, const pbn_plan& plan, const Grp& gr, const std::vector<uint32_t>& ins,
                     uint32_t shift, ImageBuild* B) {
    const size_t q = ins.size();
    if (q > 24) return fail(PBN_ETOOBIG, "group with %zu inputs (max 24)", q);
    std::vector<int> inpos(B->n, -1);
    const uint32_t in_chunk = (uint32_t)(B->inrec.size() / 4);
    for (size_t b = 0; b < q; ++b) {
        const uint32_t ps = plan.pos[ins[b]];
        if (ps == UINT32_MAX) return fail(PBN_EINVAL, "input %u of a retained node was removed", ins[b]);
        inpos[ins[b]] = (int)b;
        B->inrec.push_back(input_record(ps, b));
    }
    while (B->inrec.size() % 4) B->inrec.push_back(B->W32 << 7); /* the always-zero row */
    std::vector<uint32_t> radix(gr.nodes.size(), 0);
    uint64_t prod = 1;
    pbn_img_group G{};
    G.mul_first = (uint32_t)B->mrec.size();
    for (size_t i = 0; i < gr.nodes.size(); ++i) {
        const uint32_t v = gr.nodes[i];
        if (g.node[v].size() < 2) continue;
        radix[i] = (uint32_t)prod;
        add_choice(g, v, (uint32_t)prod, B);
        prod *= g.node[v].size();
        if (prod > (UINT64_C(1) << 30)) return fail(PBN_ETOOBIG, "group with too many combined functions");
    }
    const uint32_t width = (uint32_t)gr.nodes.size();
    const uint32_t l2w = log2_entry_bits(width);
    const uint64_t entries = prod << q;
    const uint64_t bits = entries << l2w;
    if ((double)bits > kMaxTableBits) return fail(PBN_ETOOBIG, "merged table of %llu bits exceeds 2^30", (unsigned long long)bits);
    G.tab_off = (uint32_t)B->tables.size();
    G.in_chunk = in_chunk;
    G.q = (uint8_t)q;
    G.l2w = (uint8_t)l2w;
    G.n_mul = (uint8_t)(B->mrec.size() - G.mul_first);
    G.shift = (uint8_t)shift;
    B->grec.push_back(G);
    B->total_inputs += q;
    B->tables.resize(B->tables.size() + (size_t)((bits + 31) / 32), 0);
    uint32_t* tab = B->tables.data() + G.tab_off;
    for (uint64_t c = 0; c < prod; ++c) {
        for (uint64_t x = 0; x < (1ull << q); ++x) {
            uint32_t v_out = 0;
            for (size_t i = 0; i < width; ++i) {
                const auto& fl = g.node[gr.nodes[i]];
                const size_t j = fl.size() >= 2 ? (size_t)((c / radix[i]) % fl.size()) : 0;
                const pbn_fun& f = fl[j];
                uint64_t idx = 0;
                for (size_t b = 0; b < f.par.size(); ++b) idx |= (uint64_t)((x >> inpos[f.par[b]]) & 1u) << b;
                v_out |= (uint32_t)f.bit(idx) << i;
            }
            const uint64_t bo = ((c << q) | x) << l2w;
            tab[bo >> 5] |= v_out << (bo & 31);
        }
    }
    return PBN_OK;
}

/* Group records and everything they point to (multi records, thresholds, input
 * records, tables, split-node functions), word by word. */
int emit_groups(const pbn_net& g, const pbn_group_params& prm, const PlanParts& pp, const pbn_plan& plan,
                ImageBuild* B) {
    B->words.assign(2 * B->W32, 0u);
    for (uint32_t k = 0; k < B->W32; ++k) {
        B->words[2 * k] = (uint32_t)B->grec.size();
        B->words[2 * k + 1] = (uint32_t)B->in_word[k].size();
        for (size_t gi : B->in_word[k]) {
            const Grp& gr = pp.groups[gi];
            B->n_groups_multi += gr.multi;
            std::vector<uint32_t> ins = gr.inputs; /* sorted by state position */
            std::sort(ins.begin(), ins.end(), [&](uint32_t a, uint32_t b) { return plan.pos[a] < plan.pos[b]; });
            const bool split = gr.nodes.size() == 1 && g.node[gr.nodes[0]].size() >= 2 && ins.size() > prm.max_inputs;
            const int rc = split ? add_split_group(g, plan, gr.nodes[0], B->gshift[gi], B)
                                 : add_merged_group(g, plan, gr, ins, B->gshift[gi], B);
            if (rc) return rc;
        }
    }
    return PBN_OK;
}

/* Evaluation order for lane groups and the row-interleaved record layout.  Groups
 * are sorted by shape (split nodes first by function count, then input chunks and
 * multi-function nodes descending) so that lanes taking consecutive groups run in
 * step; within a class the groups of different output words alternate (the i-th
 * group of every word, then the (i+1)-th, ...), so those lanes OR into different
 * words instead of queueing on one address.  Group records are stored in this order,
 * and the records each group reads (input chunks, multi-function nodes, split-node
 * functions) in rows of 32 groups with a stride of 32: chunk j of group k = 32 r + l
 * sits at base_r + 32 j + l, so lanes read consecutive records (no bank conflicts).
 * Split-node functions keep their own input chunks contiguous after the rows. */
int interleave_rows(ImageBuild* B, pbn_plan* plan) {
    const size_t G = B->grec.size();
    const std::vector<pbn_img_group>& grec = B->grec;
    std::vector<uint32_t> gword(G);
    for (uint32_t k = 0; k < B->W32; ++k)
        for (uint32_t gi = B->words[2 * k]; gi < B->words[2 * k] + B->words[2 * k + 1]; ++gi) gword[gi] = k;
    auto shape = [&](uint32_t a) -> uint32_t {
        const pbn_img_group& R = grec[a];
        if (R.l2w == PBN_IMG_SPLIT) return 0x10000u - R.q;
        return 0x20000u + ((255u - (R.q + 3u) / 4u) << 8) + (255u - R.n_mul);
    };
    std::vector<uint32_t> occ(G);
    {
        std::map<std::pair<uint32_t, uint32_t>, uint32_t> seen;
        for (uint32_t a = 0; a < (uint32_t)G; ++a) occ[a] = seen[{shape(a), gword[a]}]++;
    }
    std::vector<uint32_t> idx(G);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
        const uint32_t ca = shape(a), cb = shape(b);
        if (ca != cb) return ca < cb;
        if (occ[a] != occ[b]) return occ[a] < occ[b];
        return gword[a] < gword[b];
    });
    B->n_multi_nodes = (uint32_t)B->mrec.size();
    std::vector<uint32_t> newidx(G);
    for (size_t k = 0; k < G; ++k) newidx[idx[k]] = (uint32_t)k;
    std::vector<pbn_img_group> g2(G);
    std::vector<pbn_img_multi> m2;
    std::vector<uint32_t> in2, s2;
    for (size_t r0 = 0; r0 < G; r0 += 32) {
        const size_t r1 = std::min(G, r0 + 32);
        uint32_t maxc = 0, maxm = 0, maxf = 0;
        for (size_t k = r0; k < r1; ++k) {
            const pbn_img_group& O = grec[idx[k]];
            const bool sp = O.l2w == PBN_IMG_SPLIT;
            maxc = std::max<uint32_t>(maxc, sp ? 0u : (O.q + 3u) / 4u);
            maxm = std::max<uint32_t>(maxm, O.n_mul);
            maxf = std::max<uint32_t>(maxf, sp ? O.q : 0u);
        }
        const uint32_t cb = (uint32_t)(in2.size() / 4), mb = (uint32_t)m2.size(), sb = (uint32_t)(s2.size() / 2);
        in2.resize(in2.size() + (size_t)4 * 32 * maxc, B->W32 << 7); /* padding reads the zero row */
        m2.resize(m2.size() + (size_t)32 * maxm, pbn_img_multi{0u, 0u});
        s2.resize(s2.size() + (size_t)2 * 32 * maxf, 0u);
        for (size_t k = r0; k < r1; ++k) {
            const uint32_t l = (uint32_t)(k - r0);
            const pbn_img_group& O = grec[idx[k]];
            pbn_img_group N = O;
            const bool sp = O.l2w == PBN_IMG_SPLIT;
            if (!sp) {
                N.in_chunk = cb + l;
                for (uint32_t j = 0; j < (O.q + 3u) / 4u; ++j)
                    for (uint32_t e = 0; e < 4; ++e) in2[4 * (cb + l + 32 * j) + e] = B->inrec[4 * (O.in_chunk + j) + e];
            }
            N.mul_first = mb + l;
            for (uint32_t m = 0; m < O.n_mul; ++m) m2[mb + l + 32 * m] = B->mrec[O.mul_first + m];
            if (sp) {
                N.tab_off = sb + l;
                for (uint32_t f = 0; f < O.q; ++f) {
                    s2[2 * (sb + l + 32 * f)] = B->subs[2 * (O.tab_off + f)];
                    s2[2 * (sb + l + 32 * f) + 1] = B->subs[2 * (O.tab_off + f) + 1];
                }
            }
            g2[k] = N;
        }
    }
    /* split-node functions' own chunks, contiguous after the rows */
    for (size_t i = 0; i < s2.size(); i += 2) {
        const uint32_t k = s2[i] >> 27, old = s2[i] & 0x7FFFFFFu;
        if (s2[i] == 0 && s2[i + 1] == 0) continue; /* padding record */
        const uint32_t nc = (k + 3u) / 4u, at = (uint32_t)(in2.size() / 4);
        for (uint32_t j = 0; j < nc; ++j)
            for (uint32_t e = 0; e < 4; ++e) in2.push_back(B->inrec[4 * (old + j) + e]);
        if (at >= (1u << 27)) return fail(PBN_ETOOBIG, "input records beyond 2^27 chunks");
        s2[i] = at | (k << 27);
    }
    /* the groups of each output word, for the word-by-word evaluation */
    std::vector<uint32_t> wg;
    wg.reserve(G);
    for (uint32_t k = 0; k < B->W32; ++k) {
        const uint32_t first = B->words[2 * k], cnt = B->words[2 * k + 1];
        B->words[2 * k] = (uint32_t)wg.size();
        for (uint32_t gi = first; gi < first + cnt; ++gi) wg.push_back(newidx[gi]);
    }
    B->gorder.resize(G);
    for (size_t k = 0; k < G; ++k) B->gorder[k] = (uint32_t)k | (gword[idx[k]] << 20);
    for (uint32_t v = 0; v < B->n; ++v)
        if (plan->group_of[v] != UINT32_MAX) plan->group_of[v] = newidx[plan->group_of[v]];
    B->grec.swap(g2);
    B->mrec.swap(m2);
    B->inrec.swap(in2);
    B->subs.swap(s2);
    B->wgroups.swap(wg);
    return PBN_OK;
}

/* Order of the SEL blocks: a trajectory's choice row holds block i's four choice
 * bytes in word i, and the lanes that take the 32 groups of a row read their nodes'
 * choices together.  Row by row, each block not yet placed goes to a shared-memory
 * bank (word mod 32) that no other block of the row uses, while the banks' word
 * counts allow; the draws and slots only move with their blocks. */
void place_sel_blocks(ImageBuild* B) {
    if (B->selblk.size() <= 32) return;
    const uint32_t ns = (uint32_t)B->selblk.size();
    std::vector<int> bank(ns, -1);
    std::vector<uint32_t> cap(32);
    for (uint32_t b = 0; b < 32; ++b) cap[b] = ns / 32 + (b < ns % 32 ? 1u : 0u);
    auto place = [&](uint32_t blk, uint32_t used) {
        int best = -1;
        for (int b = 0; b < 32; ++b) {
            if (!cap[b]) continue;
            if (best < 0) {
                best = b;
                continue;
            }
            const bool fb = !((used >> b) & 1u), fbest = !((used >> best) & 1u);
            if (fb != fbest ? fb : cap[b] > cap[best]) best = b;
        }
        bank[blk] = best;
        cap[best]--;
        return 1u << best;
    };
    const size_t G = B->grec.size();
    for (size_t r0 = 0; r0 < G; r0 += 32) {
        const size_t r1 = std::min(G, r0 + 32);
        uint32_t used = 0;
        std::vector<uint32_t> fresh;
        for (size_t k = r0; k < r1; ++k)
            for (uint32_t m = 0; m < B->grec[k].n_mul; ++m) {
                const uint32_t blk = B->mrec[B->grec[k].mul_first + 32u * m].ch_off >> 2;
                if (bank[blk] >= 0) used |= 1u << bank[blk];
                else fresh.push_back(blk);
            }
        for (uint32_t blk : fresh) used |= bank[blk] >= 0 ? 1u << bank[blk] : place(blk, used);
    }
    for (uint32_t i = 0; i < ns; ++i)
        if (bank[i] < 0) place(i, 0u);
    std::vector<uint32_t> next(32), newpos(ns);
    std::iota(next.begin(), next.end(), 0u);
    for (uint32_t i = 0; i < ns; ++i) {
        newpos[i] = next[bank[i]];
        next[bank[i]] += 32;
    }
    std::vector<uint32_t> sb2(ns), ss2(B->selslot.size());
    for (uint32_t i = 0; i < ns; ++i) sb2[newpos[i]] = B->selblk[i];
    for (uint32_t s = 0; s < 4 * ns; ++s) {
        const uint32_t s2n = 4 * newpos[s >> 2] + (s & 3u);
        for (uint32_t e = 0; e < 4; ++e) ss2[B->slot_rec(s2n) + e] = B->selslot[B->slot_rec(s) + e];
    }
    for (pbn_img_multi& M : B->mrec)
        if (M.radix != 0) M.ch_off = 4 * newpos[M.ch_off >> 2] + (M.ch_off & 3u);
    B->selblk.swap(sb2);
    B->selslot.swap(ss2);
}

/* Header, section offsets (16-byte aligned) and the image bytes; decides whether the
 * tables are staged in shared memory with the specs (within the budget). */
int assemble_image(const pbn_net& g, const pbn_group_params& prm, const ImageBuild& B, pbn_plan* plan) {
    std::vector<uint64_t> ret(B.W, 0);
    for (uint32_t v = 0; v < B.n; ++v)
        if (g.retained[v]) ret[v >> 6] |= 1ull << (v & 63);
    pbn_img_header H{};
    H.magic = PBN_IMG_MAGIC;
    H.n = B.n;
    H.W = B.W;
    H.W32 = B.W32;
    H.n_groups = (uint32_t)B.grec.size();
    H.n_multi = (uint32_t)B.mrec.size();
    H.n_sel = (uint32_t)B.selblk.size();
    H.P = (uint32_t)pbn::pert_threshold(g.p);
    H.semantics = prm.semantics;
    H.sampler = prm.sampler;
    size_t off = align16(sizeof(pbn_img_header));
    H.off_words = (uint32_t)off; off = align16(off + B.words.size() * 4);
    H.off_groups = (uint32_t)off; off = align16(off + B.grec.size() * sizeof(pbn_img_group));
    H.off_multi = (uint32_t)off; off = align16(off + B.mrec.size() * sizeof(pbn_img_multi));
    H.off_selslot = (uint32_t)off; off = align16(off + B.selslot.size() * 4);
    H.off_thr = (uint32_t)off; off = align16(off + B.thr.size() * 4);
    H.off_inputs = (uint32_t)off; off = align16(off + B.inrec.size() * 4);
    H.off_selblk = (uint32_t)off; off = align16(off + B.selblk.size() * 4);
    H.off_gorder = (uint32_t)off; off = align16(off + B.gorder.size() * 4);
    H.off_wgroups = (uint32_t)off; off = align16(off + B.wgroups.size() * 4);
    H.off_subs = (uint32_t)off; off = align16(off + B.subs.size() * 4);
    H.off_tables = (uint32_t)off; off = align16(off + B.tables.size() * 4);
    H.off_ret = (uint32_t)off; off = align16(off + ret.size() * 8);
    H.off_pos = (uint32_t)off; off = align16(off + plan->pos.size() * 4);
    H.off_geo = (uint32_t)off; off = align16(off + 64 * 8);
    if (off >= (UINT64_C(1) << 31)) return fail(PBN_ETOOBIG, "device image of %zu bytes", off);
    H.image_bytes = (uint32_t)off;
    const uint64_t budget = prm.smem_budget ? prm.smem_budget : 192 * 1024;
    H.tables_in_smem = H.off_ret <= budget ? 1u : 0u;
    H.stage_bytes = H.tables_in_smem ? H.off_ret : H.off_tables;
    if (H.stage_bytes > budget) return fail(PBN_ETOOBIG, "plan specs of %u bytes exceed the shared-memory budget", H.stage_bytes);

    plan->image.assign(off, 0);
    uint8_t* img = plan->image.data();
    auto put = [&](uint32_t at, const void* src, size_t bytes) {
        if (bytes) memcpy(img + at, src, bytes);
    };
    memcpy(img, &H, sizeof(H));
    put(H.off_words, B.words.data(), B.words.size() * 4);
    put(H.off_groups, B.grec.data(), B.grec.size() * sizeof(pbn_img_group));
    put(H.off_multi, B.mrec.data(), B.mrec.size() * sizeof(pbn_img_multi));
    put(H.off_selslot, B.selslot.data(), B.selslot.size() * 4);
    put(H.off_thr, B.thr.data(), B.thr.size() * 4);
    put(H.off_inputs, B.inrec.data(), B.inrec.size() * 4);
    put(H.off_selblk, B.selblk.data(), B.selblk.size() * 4);
    put(H.off_gorder, B.gorder.data(), B.gorder.size() * 4);
    put(H.off_wgroups, B.wgroups.data(), B.wgroups.size() * 4);
    put(H.off_subs, B.subs.data(), B.subs.size() * 4);
    put(H.off_ret, ret.data(), ret.size() * 8);
    put(H.off_pos, plan->pos.data(), plan->pos.size() * 4);
    uint64_t geo[64];
    geometric_thresholds(H.P, geo);
    put(H.off_geo, geo, sizeof(geo));
    put(H.off_tables, B.tables.data(), B.tables.size() * 4);
    plan->hdr = H;
    plan->per_traj_smem = 4 * (2 * (B.W32 + 1) + (H.n_sel | 1u));
    return PBN_OK;
}

/* pbn_plan_info, with the algorithmic work of one trajectory-step (the roofline's
 * per-unit figure): Philox4x32-10 blocks at 56 ops, the expected perturbation levels
 * (or the geometric sampler's block per word pair), and, weighted by the probability
 * of a non-perturbed step, the SEL blocks, thresholds, gathers and lookups. */
void fill_info(const pbn_net& g, const pbn_group_params& prm, const PlanParts& pp, const ImageBuild& B,
               pbn_plan* plan) {
    const pbn_img_header& H = plan->hdr;
    pbn_plan_info& I = plan->info;
    memset(&I, 0, sizeof(I));
    I.n = B.n;
    for (uint32_t v = 0; v < B.n; ++v) I.n_retained += g.retained[v];
    I.n_groups = H.n_groups;
    I.n_groups_multi = B.n_groups_multi;
    I.state_words = B.W32 / 2;
    I.n_sel_blocks = H.n_sel;
    I.m_lower_bound = pp.m_lower;
    I.m_found = pp.m_found;
    I.sum_weights = pp.sum_w;
    I.table_bytes = B.tables.size() * 4;
    I.image_bytes = H.image_bytes;
    I.stage_bytes = H.stage_bytes;
    I.tables_in_smem = H.tables_in_smem;
    I.total_inputs = (uint32_t)B.total_inputs;
    I.n_multi = B.n_multi_nodes;
    I.n_split = B.n_split;
    I.semantics = prm.semantics;
    I.sampler = prm.sampler;
    I.total_thresholds = (uint32_t)B.thr.size();
    const uint32_t n = B.n, W = B.W;
    const double pe = (double)H.P / 4294967296.0;
    double blocks = 0.0;
    if (H.P) {
        for (uint32_t w = 0; w < W; ++w) {
            const uint32_t k = (w == W - 1 && (n & 63u)) ? (n & 63u) : 64u;
            for (int h = 0; h < 16; ++h) blocks += 1.0 - std::pow(1.0 - std::ldexp(1.0, -2 * h), (double)k);
        }
    }
    double pert = blocks * (56.0 + 12.0) + 4.0;
    if (prm.sampler == PBN_PERT_GEOMETRIC) /* one block per word pair, a 64-bit compare per word */
        pert = H.P ? 56.0 * (double)((W + 1) / 2) + 4.0 * (double)W + 4.0 : 4.0;
    const double nonpert = 56.0 * H.n_sel + 2.0 * (double)B.thr.size() + (double)B.n_multi_nodes +
                           3.0 * (double)B.total_inputs + 5.0 * (double)(H.n_groups + B.n_split) +
                           2.0 * (double)(B.W32 / 2);
    I.ops_per_step = pert + std::pow(1.0 - pe, (double)n) * nonpert + 8.0;
}

int build_plan(const pbn_net& g, const pbn_group_params& prm, pbn_plan* plan) {
    PlanParts pp;
    partition(g, prm, &pp);
    ImageBuild B;
    B.n = g.n;
    B.W = (g.n + 63) / 64;
    pack_words(pp, &B);
    place_nodes(pp, B, plan);
    sel_blocks(g, &B);
    int rc = emit_groups(g, prm, pp, *plan, &B);
    if (rc == PBN_OK) rc = interleave_rows(&B, plan);
    if (rc != PBN_OK) return rc;
    place_sel_blocks(&B);
    rc = assemble_image(g, prm, B, plan);
    if (rc != PBN_OK) return rc;
    fill_info(g, prm, pp, B, plan);
    return PBN_OK;
}

}  // namespace

extern "C" void pbn_group_params_default(pbn_group_params* prm) {
    if (!prm) return;
    memset(prm, 0, sizeof(*prm));
    prm->mode = PBN_PLAN_GROUPED;
    prm->max_inputs = 8;
    prm->max_width = 32;
    prm->theta = 65536.0;
    prm->smem_budget = 192 * 1024;
}

extern "C" int pbn_group(const pbn_net* net, const pbn_group_params* prm_in, pbn_plan** out) {
    if (!net || !out) return fail(PBN_EINVAL, "pbn_group: NULL argument");
    *out = nullptr;
    pbn_group_params prm;
    pbn_group_params_default(&prm);
    if (prm_in) prm = *prm_in;
    if (prm.mode != PBN_PLAN_GROUPED && prm.mode != PBN_PLAN_PLAIN)
        return fail(PBN_EINVAL, "pbn_group: unknown mode %u", prm.mode);
    if (prm.max_inputs < 1 || prm.max_inputs > 24 || prm.max_width < 1 || prm.max_width > 32 ||
        !(prm.theta >= 1.0) || (prm.smem_budget && prm.smem_budget < 1024) ||
        (prm.semantics != PBN_SEM_EQ1 && prm.semantics != PBN_SEM_NODEWISE) ||
        (prm.sampler != PBN_PERT_BITSLICED && prm.sampler != PBN_PERT_GEOMETRIC))
        return fail(PBN_EINVAL, "pbn_group: parameter out of range");
    try {
        pbn_plan* plan = new pbn_plan();
        int rc = build_plan(*net, prm, plan);
        if (rc) { delete plan; return rc; }
        *out = plan;
        return PBN_OK;
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_group: out of memory");
    }
}

pbn_plan::~pbn_plan() { pbn::jit_free(jit); }

extern "C" void pbn_plan_free(pbn_plan* plan) { delete plan; }

extern "C" int pbn_plan_info_get(const pbn_plan* plan, pbn_plan_info* out) {
    if (!plan || !out) return fail(PBN_EINVAL, "pbn_plan_info_get: NULL argument");
    *out = plan->info;
    return PBN_OK;
}

extern "C" int pbn_plan_image(const pbn_plan* plan, void* dst, size_t cap) {
    if (!plan || !dst) return fail(PBN_EINVAL, "pbn_plan_image: NULL argument");
    if (cap < plan->image.size()) return fail(PBN_EINVAL, "pbn_plan_image: need %zu bytes", plan->image.size());
    memcpy(dst, plan->image.data(), plan->image.size());
    return PBN_OK;
}

extern "C" int pbn_plan_layout(const pbn_plan* plan, uint32_t* pos) {
    if (!plan || !pos) return fail(PBN_EINVAL, "pbn_plan_layout: NULL argument");
    memcpy(pos, plan->pos.data(), plan->pos.size() * 4);
    return PBN_OK;
}

extern "C" int pbn_plan_groups(const pbn_plan* plan, uint32_t* group_of) {
    if (!plan || !group_of) return fail(PBN_EINVAL, "pbn_plan_groups: NULL argument");
    memcpy(group_of, plan->group_of.data(), plan->group_of.size() * 4);
    return PBN_OK;
}

/* ------------------------------------------------------------------------- */
/* Two-state Markov chain estimate (Sec. 4.2)                                 */
/* ------------------------------------------------------------------------- */
namespace {
/* Standard normal quantile: bisection on Phi(x) = erfc(-x / sqrt 2) / 2 to bracket
 * the root, then Newton steps with the normal density. */
double norm_quantile(double prob) {
    double lo = -40.0, hi = 40.0;
    auto Phi = [](double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); };
    for (int it = 0; it < 80; ++it) {
        double mid = 0.5 * (lo + hi);
        if (Phi(mid) < prob) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) {
        double pdf = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
        if (pdf <= 0.0) break;
        x -= (Phi(x) - prob) / pdf;
    }
    return x;
}
}  // namespace

extern "C" int pbn_estimate(const uint64_t counts[5], uint64_t n_traj, uint64_t burn_in_used, double r,
                            double s, double eps, pbn_estimate_out* out) {
    if (!counts || !out || !(r > 0.0) || !(s > 0.0 && s < 1.0) || !(eps > 0.0) || n_traj == 0)
        return fail(PBN_EINVAL, "pbn_estimate: argument out of range");
    const uint64_t V = counts[0], n00 = counts[1], n01 = counts[2], n10 = counts[3], n11 = counts[4];
    pbn_estimate_out o;
    memset(&o, 0, sizeof(o));
    o.L = n00 + n01 + n10 + n11 + n_traj;
    o.alpha = (n00 + n01) ? (double)n01 / (double)(n00 + n01) : NAN;
    o.beta = (n10 + n11) ? (double)n10 / (double)(n10 + n11) : NAN;
    o.pi = (double)V / (double)o.L;
    o.z = norm_quantile((1.0 + s) / 2.0);
    o.m_star = UINT64_MAX;
    o.n_star = UINT64_MAX;
    o.var = NAN;
    o.n_star_real = NAN;
    const double a = o.alpha, b = o.beta;
    if (!std::isnan(a) && !std::isnan(b) && a + b > 0.0) {
        o.defined = (a > 0.0 && b > 0.0) ? 1 : 0;
        const double lam = std::fabs(1.0 - a - b);
        if (lam == 0.0) {
            o.m_star = 1;
        } else if (lam < 1.0) {
            double m = std::ceil(std::log(eps * (a + b) / std::max(a, b)) / std::log(lam));
            o.m_star = m < 1.0 ? 1 : (uint64_t)m;
        }
        const double ab = a * b * (2.0 - a - b) / ((a + b) * (a + b) * (a + b));
        o.n_star_real = ab * (o.z / r) * (o.z / r);
        o.n_star = (uint64_t)std::ceil(o.n_star_real);
        o.var = ab / (double)o.L;
    }
    o.done = (o.defined && o.m_star != UINT64_MAX && o.L >= o.n_star && burn_in_used >= o.m_star) ? 1 : 0;
    *out = o;
    return PBN_OK;
}
