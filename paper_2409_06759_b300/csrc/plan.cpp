// plan.cpp -- parser and TTGT planner for contraction lists.
//
// Grammar (one statement per line, '#' comment):
//   OUT[idx].. (=|+=|-=) [factor] [P(pq)|P(p/qr)]... A[idx].. [* B[idx]..]
// This is the text form of the "Contraction" class of arxiv 2409.06759
// Sec. II C (factor, permutation operators, tensors, output); as in the
// paper's Fig. algo:remove, only binary contractions are accepted.
#include "plan.h"

#include <algorithm>
#include <array>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <sstream>

namespace ccb {

// bytes of an operand's split planes: bf16 planes [nplanes][R][Kp]; the six
// exact slices are followed by one int32 row exponent per row
static int64_t planes_bytes(int64_t R, int64_t Kp, int nplanes) {
    return R * Kp * 2 * nplanes + (nplanes == 6 ? R * 4 : 0);
}

static const char *kBlockNames[6] = {"oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv"};

void integral_block_dims(int o, int v, int block, int64_t ext[4]) {
    for (int d = 0; d < 4; d++) ext[d] = kBlockNames[block][d] == 'o' ? o : v;
}

namespace {

constexpr int64_t kAlign = 256;
int64_t align_up(int64_t x, int64_t a = kAlign) { return (x + a - 1) / a * a; }

struct Ref {
    std::string name;
    std::vector<int> letters;   // letter ids in written order
    std::vector<std::array<int, 2>> pairs;   // declared antisymmetric pairs "(pq)": positions in letters
};

struct Stmt {
    int line = 0;
    Ref out;
    int op = 0;                 // 0 '=', +1 '+=', -1 '-='
    double factor = 1.0;
    std::vector<std::pair<std::vector<int>, bool>> perms;  // letters, slash form
    std::vector<Ref> rhs;
};

struct Parser {
    const std::string &s;
    size_t p = 0;
    std::vector<std::string> &tokens;   // letter id -> token
    std::vector<char> &spaces;
    std::string err;
    Parser(const std::string &line, std::vector<std::string> &t, std::vector<char> &sp)
        : s(line), tokens(t), spaces(sp) {}
    void ws() {
        while (p < s.size() && std::isspace((unsigned char)s[p])) p++;
    }
    bool eat(char c) {
        ws();
        if (p < s.size() && s[p] == c) { p++; return true; }
        return false;
    }
    bool at_end() { ws(); return p >= s.size(); }
    int letter_id(const std::string &tok) {
        for (size_t k = 0; k < tokens.size(); k++)
            if (tokens[k] == tok) return (int)k;
        char sp = 0;
        if (tok.size() == 1) {
            char c = tok[0];
            if (c >= 'a' && c <= 'h') sp = 'v';
            else if (c >= 'i' && c <= 'n') sp = 'o';
        } else if (tok[0] == 'p') sp = 'v';
        else if (tok[0] == 'h') sp = 'o';
        if (!sp) { err = "index '" + tok + "' is neither occupied (i..n, h<k>) nor virtual (a..h, p<k>)"; return -1; }
        tokens.push_back(tok);
        spaces.push_back(sp);
        return (int)tokens.size() - 1;
    }
    // reads [a-z][0-9]* tokens until the closing bracket
    bool letters_until(char close, std::vector<int> &out, std::vector<int> *slash_pos = nullptr,
                       std::vector<std::array<int, 2>> *pairs = nullptr) {
        int open = -1;   // position where a "(pq)" pair started
        for (;;) {
            ws();
            if (p >= s.size()) { err = "missing closing bracket"; return false; }
            char c = s[p];
            if (c == close) {
                if (open >= 0) { err = "unclosed '(' in index list"; return false; }
                p++;
                return true;
            }
            if (c == ',') { p++; continue; }
            if (c == '(' && pairs) {
                if (open >= 0) { err = "nested '(' in index list"; return false; }
                open = (int)out.size();
                p++;
                continue;
            }
            if (c == ')' && pairs) {
                if (open < 0 || (int)out.size() - open != 2) {
                    err = "'(..)' must enclose exactly two indices";
                    return false;
                }
                pairs->push_back({open, open + 1});
                open = -1;
                p++;
                continue;
            }
            if (c == '/' && slash_pos) { slash_pos->push_back((int)out.size()); p++; continue; }
            if (!(c >= 'a' && c <= 'z')) { err = std::string("unexpected character '") + c + "' in index list"; return false; }
            std::string tok(1, c);
            p++;
            while (p < s.size() && std::isdigit((unsigned char)s[p])) tok += s[p++];
            int id = letter_id(tok);
            if (id < 0) return false;
            out.push_back(id);
        }
    }
    bool ref(Ref &r) {
        ws();
        size_t q = p;
        while (p < s.size() && (std::isalnum((unsigned char)s[p]) || s[p] == '_')) p++;
        if (p == q || std::isdigit((unsigned char)s[q])) { err = "expected a tensor name"; return false; }
        r.name = s.substr(q, p - q);
        bool any = false;
        while (eat('[')) {
            if (!letters_until(']', r.letters, nullptr, &r.pairs)) return false;
            any = true;
        }
        if (!any) { err = "tensor '" + r.name + "' has no index brackets"; return false; }
        return true;
    }
    bool number(double &x) {
        ws();
        const char *b = s.c_str() + p;
        char *e = nullptr;
        x = std::strtod(b, &e);
        if (e == b) return false;
        p += (size_t)(e - b);
        ws();
        if (p + 1 < s.size() && s[p] == '/' && std::isdigit((unsigned char)s[p + 1])) {
            p++;
            const char *b2 = s.c_str() + p;
            double d = std::strtod(b2, &e);
            p += (size_t)(e - b2);
            if (d == 0.0) { err = "division by zero in factor"; return false; }
            x /= d;
        }
        return true;
    }
};

bool parse_stmt(const std::string &line, Stmt &st, std::vector<std::string> &tokens,
                std::vector<char> &spaces, std::string &err) {
    Parser P(line, tokens, spaces);
    if (!P.ref(st.out)) { err = P.err; return false; }
    P.ws();
    if (P.s.compare(P.p, 2, "+=") == 0) { st.op = 1; P.p += 2; }
    else if (P.s.compare(P.p, 2, "-=") == 0) { st.op = -1; P.p += 2; }
    else if (P.eat('=')) st.op = 0;
    else { err = "expected '=', '+=' or '-='"; return false; }
    st.factor = 1.0;
    P.ws();
    // factor: a number (optionally a/b), or a bare sign
    if (P.p < P.s.size() && (P.s[P.p] == '-' || P.s[P.p] == '+')) {
        bool neg = P.s[P.p] == '-';
        size_t q = P.p + 1;
        while (q < P.s.size() && std::isspace((unsigned char)P.s[q])) q++;
        P.p = q;
        double x = 1.0;
        if (q < P.s.size() && (std::isdigit((unsigned char)P.s[q]) || P.s[q] == '.')) {
            if (!P.number(x)) { err = P.err.empty() ? "bad factor" : P.err; return false; }
        }
        st.factor = neg ? -x : x;
    } else if (P.p < P.s.size() && (std::isdigit((unsigned char)P.s[P.p]) || P.s[P.p] == '.')) {
        double x;
        if (!P.number(x)) { err = P.err.empty() ? "bad factor" : P.err; return false; }
        st.factor = x;
    }
    P.eat('*');
    // permutation operators
    for (;;) {
        P.ws();
        if (P.p + 1 < P.s.size() && P.s[P.p] == 'P' && P.s[P.p + 1] == '(') {
            P.p += 2;
            std::vector<int> ls, slash;
            if (!P.letters_until(')', ls, &slash)) { err = P.err; return false; }
            bool sl = !slash.empty();
            if (sl && (slash.size() != 1 || slash[0] != 1 || ls.size() < 3)) {
                err = "permutation operator must be P(pq) or P(p/qr..)";
                return false;
            }
            if (!sl && ls.size() != 2) { err = "permutation operator P(pq) needs exactly two indices"; return false; }
            st.perms.push_back({ls, sl});
            P.eat('*');
        } else {
            break;
        }
    }
    Ref a;
    if (!P.ref(a)) { err = P.err; return false; }
    st.rhs.push_back(a);
    if (P.eat('*')) {
        Ref b;
        if (!P.ref(b)) { err = P.err; return false; }
        st.rhs.push_back(b);
    }
    if (!P.at_end()) {
        err = "unexpected text after the contraction (only binary contractions are accepted)";
        return false;
    }
    return true;
}

struct Perm {
    double sign;
    std::map<int, int> sigma;   // letter -> letter (identity when absent)
    int at(int l) const {
        auto it = sigma.find(l);
        return it == sigma.end() ? l : it->second;
    }
};

// Expands a product of permutation operators into signed relabellings.  A
// relabelling sigma acts as (sigma X)(idx) = X(idx'), idx'(l) = idx(sigma(l)).
std::vector<Perm> expand_perms(const std::vector<std::pair<std::vector<int>, bool>> &ps) {
    std::vector<Perm> terms(1, Perm{1.0, {}});
    for (auto &pp : ps) {
        std::vector<Perm> ops;
        ops.push_back(Perm{1.0, {}});
        const auto &ls = pp.first;
        if (!pp.second) {
            ops.push_back(Perm{-1.0, {{ls[0], ls[1]}, {ls[1], ls[0]}}});
        } else {
            for (size_t k = 1; k < ls.size(); k++) ops.push_back(Perm{-1.0, {{ls[0], ls[k]}, {ls[k], ls[0]}}});
        }
        std::vector<Perm> nt;
        for (auto &t : terms)
            for (auto &op : ops) {
                Perm c{t.sign * op.sign, {}};
                std::set<int> keys;
                for (auto &kv : t.sigma) keys.insert(kv.first);
                for (auto &kv : op.sigma) keys.insert(kv.first);
                for (int l : keys) {
                    int m = t.at(op.at(l));
                    if (m != l) c.sigma[l] = m;
                }
                nt.push_back(c);
            }
        terms.swap(nt);
    }
    return terms;
}

struct Planner {
    Plan &plan;
    int o, v;
    std::string err;
    std::map<std::string, int> by_name;
    std::vector<bool> initialized;
    int64_t scratch_need = 0;       // arena bytes of the current statement
    int64_t cache_need = 0;         // static split planes
    int64_t interm_need = kAlign;   // [status word][intermediates...] at the start of the workspace
    int64_t splits_need = 0;        // planes of non-static split operands, kept for reuse within a residual
    bool mixed_all = false;
    bool uniform = false;          // uniform steps: routes fixed by the statement's form, not its extents
    bool kcat_declined = false;    // set by plan_kcat when some members run cheaper one by one
    std::vector<char> kcat_keep;   // with it: the members that still gain from merging
    std::vector<int> version;       // per tensor: number of statements that wrote it so far

    // one split of a tensor version into planes, reusable by later steps
    struct SplitRec {
        int tensor, version, np;
        SplitDesc d;
        int64_t off;
    };
    std::vector<SplitRec> splits;

    static bool same_grp(const Grp &a, const Grp &b) {
        if (a.nd != b.nd) return false;
        for (int k = 0; k < a.nd; k++)
            if (a.ext[k] != b.ext[k] || a.str[k] != b.str[k]) return false;
        return true;
    }
    // offset of the planes (split-region relative) and whether they already exist
    int64_t split_slot(int tensor, const SplitDesc &d, bool &exists) {
        const int ver = version[tensor];
        for (auto &r : splits)
            if (r.tensor == tensor && r.version == ver && r.np == d.nplanes && r.d.R == d.R && r.d.K == d.K &&
                r.d.cplx == d.cplx && r.d.conj == d.conj &&
                r.d.Rp == d.Rp && r.d.Kp == d.Kp && same_grp(r.d.gr, d.gr) && same_grp(r.d.gk, d.gk)) {
                exists = true;
                return r.off;
            }
        exists = false;
        SplitRec r{tensor, ver, d.nplanes, d, splits_need};
        splits_need += align_up(planes_bytes(d.Rp, d.Kp, d.nplanes));
        splits.push_back(r);
        return r.off;
    }

    explicit Planner(Plan &pl) : plan(pl), o(pl.o), v(pl.v), cplx(pl.dtype == 1), esz(pl.dtype == 1 ? 16 : 8) {}
    // 'o', 'v': orbital indices; 'O', 'V': packed pairs p < q of them
    int64_t space_extent(char sp) const {
        return sp == 'o' ? o : sp == 'v' ? v : sp == 'O' ? (int64_t)o * (o - 1) / 2 : (int64_t)v * (v - 1) / 2;
    }
    const bool cplx;            // complex double elements (interleaved re, im)
    const int64_t esz;          // bytes per element

    // complex-element strides -> double strides
    static Grp dbl(Grp g) {
        for (int k = 0; k < g.nd; k++) g.str[k] *= 2;
        return g;
    }
    // appends the re/im component as the fastest digit of a double-addressed group
    bool add_component(Grp &g) {
        if (g.nd >= 6) { err = "more than five indices in one matrix dimension of a complex contraction"; return false; }
        g.ext[g.nd] = 2;
        g.str[g.nd] = 1;
        g.nd++;
        return true;
    }

    int add_tensor(const std::string &name, TKind k, const std::vector<char> &sp, int slot) {
        Tensor t;
        t.name = name;
        t.kind = k;
        t.spaces = sp;
        t.slot = slot;
        int64_t e = 1;
        t.ext.resize(sp.size());
        t.str.resize(sp.size());
        for (size_t d = 0; d < sp.size(); d++) t.ext[d] = space_extent(sp[d]);
        for (int d = (int)sp.size() - 1; d >= 0; d--) { t.str[d] = e; e *= t.ext[d]; }
        t.elems = e;
        if (k == TKind::INTERM) { t.ws_off = interm_need; interm_need += align_up(e * esz); }
        plan.tensors.push_back(t);
        version.push_back(0);
        initialized.push_back(k != TKind::RES && k != TKind::INTERM);
        by_name[name] = (int)plan.tensors.size() - 1;
        return (int)plan.tensors.size() - 1;
    }

    bool resolve(const Ref &r, bool is_out, int op, const std::vector<char> &lsp, View &vw) {
        const std::string &nm = r.name;
        const int rank = (int)r.letters.size();
        std::set<int> uniq(r.letters.begin(), r.letters.end());
        if ((int)uniq.size() != rank) { err = "repeated index in " + nm; return false; }
        auto is_amp = [](const std::string &x) {
            return x == "t" || x == "T" || x == "T1" || x == "T2" || x == "T3" || x == "t1" || x == "t2" || x == "t3";
        };
        auto is_res = [](const std::string &x) {
            return x == "R" || x == "r" || x == "R1" || x == "R2" || x == "R3" || x == "r1" || x == "r2" || x == "r3";
        };
        if (is_amp(nm) || is_res(nm)) {
            bool amp = is_amp(nm);
            if (rank % 2 || rank < 2 || rank > 6) { err = nm + " needs 2, 4 or 6 indices"; return false; }
            int lvl = rank / 2;
            if (nm.size() == 2 && nm[1] - '0' != lvl) { err = nm + " has the wrong number of indices"; return false; }
            std::vector<int> occ, vir;
            for (int l : r.letters) (lsp[l] == 'o' ? occ : vir).push_back(l);
            if ((int)occ.size() != lvl) { err = nm + " needs equal numbers of occupied and virtual indices"; return false; }
            std::string key = std::string(amp ? "T" : "R") + char('0' + lvl);
            if (amp && is_out) { err = "amplitudes are inputs and cannot be assigned"; return false; }
            if (!amp && !is_out) { err = "residual tensors are outputs only"; return false; }
            int id;
            auto it = by_name.find(key);
            if (it == by_name.end()) {
                std::vector<char> sp(lvl, 'o');
                sp.insert(sp.end(), lvl, 'v');
                id = add_tensor(key, amp ? TKind::AMP : TKind::RES, sp, lvl);
            } else {
                id = it->second;
            }
            if (amp) plan.amp_used[lvl] = true; else plan.res_used[lvl] = true;
            vw.tensor = id;
            vw.idx = occ;
            vw.idx.insert(vw.idx.end(), vir.begin(), vir.end());
        } else if (nm == "V" || nm == "v") {
            if (is_out) { err = "integrals are inputs and cannot be assigned"; return false; }
            if (rank != 4) { err = "V needs four indices <pq||rs> = V[pq][rs]"; return false; }
            char s[4];
            for (int d = 0; d < 4; d++) s[d] = lsp[r.letters[d]];
            bool found = false;
            // <pq||rs> = -<qp||rs> = -<pq||sr> = conj(<rs||pq>): search the canonical block
            for (int bk = 0; bk < 2 && !found; bk++)
                for (int bs = 0; bs < 2 && !found; bs++)
                    for (int ks = 0; ks < 2 && !found; ks++) {
                        int pos[4] = {0, 1, 2, 3};
                        double sg = 1.0;
                        if (bk) { pos[0] = 2; pos[1] = 3; pos[2] = 0; pos[3] = 1; }
                        if (bs) { std::swap(pos[0], pos[1]); sg = -sg; }
                        if (ks) { std::swap(pos[2], pos[3]); sg = -sg; }
                        char pat[5] = {s[pos[0]], s[pos[1]], s[pos[2]], s[pos[3]], 0};
                        for (int b = 0; b < 6; b++)
                            if (!std::strcmp(pat, kBlockNames[b])) {
                                std::string key = std::string("V_") + kBlockNames[b];
                                auto it = by_name.find(key);
                                int id = it == by_name.end()
                                             ? add_tensor(key, TKind::INTEGRAL, std::vector<char>(pat, pat + 4), b)
                                             : it->second;
                                vw.tensor = id;
                                vw.idx.resize(4);
                                for (int d = 0; d < 4; d++) vw.idx[d] = r.letters[pos[d]];
                                vw.sign = sg;
                                vw.conj = bk != 0;
                                found = true;
                                break;
                            }
                    }
            if (!found) { err = "internal: no canonical integral block"; return false; }
        } else {
            std::vector<char> sp;
            for (int l : r.letters) sp.push_back(lsp[l]);
            auto it = by_name.find(nm);
            int id;
            if (it == by_name.end()) {
                if (!is_out || op != 0) {
                    err = "intermediate '" + nm + "' is used before a defining '=' statement";
                    return false;
                }
                id = add_tensor(nm, TKind::INTERM, sp, 0);
            } else {
                id = it->second;
                const Tensor &t = plan.tensors[id];
                // (internal '%' names: packed operands, which may be integral inputs)
                if (t.kind != TKind::INTERM && nm[0] != '%') { err = "name '" + nm + "' is reserved"; return false; }
                if (t.spaces != sp) { err = "index spaces of '" + nm + "' differ from its definition"; return false; }
            }
            vw.tensor = id;
            vw.idx = r.letters;
        }
        const Tensor &t = plan.tensors[vw.tensor];
        vw.ext = t.ext;
        vw.str = t.str;
        return true;
    }

    struct Fuse {
        bool ok = true;
        std::vector<int> order;     // letters, outermost first (extent-1 letters last)
        int64_t stride = 0, extent = 1;
    };

    // Can the letters `grp` of view `vw` be addressed as one index with a single
    // stride?  The only candidate order is by decreasing stride.
    static Fuse fusable(const View &vw, const std::set<int> &grp) {
        Fuse f;
        std::vector<int> dims, ones;
        for (size_t d = 0; d < vw.idx.size(); d++)
            if (grp.count(vw.idx[d])) (vw.ext[d] > 1 ? dims : ones).push_back((int)d);
        std::sort(dims.begin(), dims.end(), [&](int x, int y) { return vw.str[x] > vw.str[y]; });
        for (size_t t = 0; t + 1 < dims.size(); t++)
            if (vw.str[dims[t]] != vw.str[dims[t + 1]] * vw.ext[dims[t + 1]]) f.ok = false;
        for (int d : dims) { f.order.push_back(vw.idx[d]); f.extent *= vw.ext[d]; }
        for (int d : ones) f.order.push_back(vw.idx[d]);
        f.stride = dims.empty() ? 1 : vw.str[dims.back()];
        return f;
    }

    static bool same_order(const View &va, const std::vector<int> &a, const View &vb, const std::vector<int> &b) {
        auto strip = [](const View &vw, const std::vector<int> &o) {
            std::vector<int> r;
            for (int l : o)
                for (size_t d = 0; d < vw.idx.size(); d++)
                    if (vw.idx[d] == l && vw.ext[d] > 1) r.push_back(l);
            return r;
        };
        return strip(va, a) == strip(vb, b);
    }

    static int64_t ext_of(const View &vw, int l) {
        for (size_t d = 0; d < vw.idx.size(); d++)
            if (vw.idx[d] == l) return vw.ext[d];
        return 1;
    }
    static int64_t str_of(const View &vw, int l) {
        for (size_t d = 0; d < vw.idx.size(); d++)
            if (vw.idx[d] == l) return vw.str[d];
        return 0;
    }

    BufRef tensor_ref(int id) const {
        const Tensor &t = plan.tensors[id];
        BufRef r;
        switch (t.kind) {
            case TKind::AMP: r.where = BufRef::AMP; r.slot = t.slot; break;
            case TKind::RES: r.where = BufRef::RES; r.slot = t.slot; break;
            case TKind::INTEGRAL: r.where = BufRef::INTEG; r.slot = t.slot; break;
            case TKind::INTERM: r.where = BufRef::WS; r.off = t.ws_off; break;
        }
        return r;
    }

    BufRef scratch(int64_t bytes) {
        BufRef r;
        r.where = BufRef::WS;
        r.slot = 1;                 // arena-relative; rebased after planning
        r.off = scratch_need;
        scratch_need += align_up(bytes);
        return r;
    }

    Grp make_grp(const std::vector<int> &letters, const View &ext_src, const View &str_src) {
        Grp g{};
        for (int l : letters) {
            if (ext_of(ext_src, l) <= 1) continue;
            if (g.nd >= 6) { err = "more than six indices in one matrix dimension"; return g; }
            g.ext[g.nd] = ext_of(ext_src, l);
            g.str[g.nd] = str_of(str_src, l);
            g.nd++;
        }
        return g;
    }

    // ACCUM step: out (view over OUT letters) = beta*out + alpha*sum_p s_p src[sigma_p]
    Step accum_step(const View &out, BufRef outref, const View &src, BufRef srcref, const std::vector<Perm> &perms,
                    double alpha, double beta) {
        Step st;
        st.kind = StepKind::ACCUM;
        st.out = outref;
        st.a = srcref;
        if ((int)perms.size() > kMaxPerms || (int)out.idx.size() > kMaxDims) {
            err = "more than " + std::to_string(kMaxPerms) + " permutation terms or " + std::to_string(kMaxDims) +
                  " indices in one statement";
            return st;
        }
        AccumDesc &d = st.acc;
        d.nd = (int)out.idx.size();
        d.nperm = (int)perms.size();
        d.total = 1;
        for (int k = 0; k < d.nd; k++) {
            d.ext[k] = out.ext[k];
            d.ostr[k] = out.str[k];
            d.total *= out.ext[k];
        }
        for (int p = 0; p < d.nperm; p++) {
            d.sign[p] = perms[p].sign;
            for (int k = 0; k < d.nd; k++) {
                // the source stride for output letter mu is that of sigma^-1(mu)
                int mu = out.idx[k];
                int pre = mu;
                for (auto &kv : perms[p].sigma)
                    if (kv.second == mu) pre = kv.first;
                d.sstr[p][k] = str_of(src, pre);
            }
        }
        d.alpha = alpha;
        d.beta = beta;
        d.cplx = cplx ? 1 : 0;
        d.conj_a = cplx && src.conj ? 1 : 0;
        st.note = "accum";
        return st;
    }

    // contiguous buffer view with the given letter order
    static View contiguous_view(const std::vector<int> &order, const View &ext_src1, const View *ext_src2 = nullptr) {
        View w;
        w.tensor = -1;
        w.idx = order;
        w.ext.resize(order.size());
        w.str.resize(order.size());
        int64_t e = 1;
        for (int d = (int)order.size() - 1; d >= 0; d--) {
            int64_t x = ext_of(ext_src1, order[d]);
            if (x <= 1 && ext_src2) x = ext_of(*ext_src2, order[d]);
            w.ext[d] = x;
            w.str[d] = e;
            e *= x;
        }
        return w;
    }

    static int64_t view_elems(const View &w) {
        int64_t e = 1;
        for (auto x : w.ext) e *= x;
        return e;
    }

    int last_out = 0;

    // The pair letters of declared pair q of a reference, in written order.
    static std::array<int, 2> pair_letters(const Ref &r, int q) {
        return {r.letters[r.pairs[q][0]], r.letters[r.pairs[q][1]]};
    }

    // A packed operand: a PACK step from view X into a new intermediate
    // [free pair][contracted pair] (static when X is an integral block).
    int pack_operand(const View &X, std::array<int, 2> fp, std::array<int, 2> kp, char sf, char sk,
                     const std::string &name, int si) {
        // <ab||ef> packed in its stored orientation is an input of its own
        const Tensor &TX = plan.tensors[X.tensor];
        if (plan.packed_vvvv && TX.kind == TKind::INTEGRAL && TX.slot == 5 && X.idx.size() == 4 &&
            X.idx[0] == fp[0] && X.idx[1] == fp[1] && X.idx[2] == kp[0] && X.idx[3] == kp[1]) {
            auto it = by_name.find("%V_vvvv_packed");
            return it != by_name.end() ? it->second
                                       : add_tensor("%V_vvvv_packed", TKind::INTEGRAL, std::vector<char>{'V', 'V'}, 6);
        }
        const int id = add_tensor(name, TKind::INTERM, std::vector<char>{sf, sk}, 0);
        initialized[id] = true;
        Step st;
        st.kind = StepKind::PACK;
        st.stmt = si;
        st.a = tensor_ref(X.tensor);
        st.out = tensor_ref(id);
        PackDesc &d = st.pk;
        d.n1 = ext_of(X, fp[0]);
        d.n2 = ext_of(X, kp[0]);
        d.P1 = d.n1 * (d.n1 - 1) / 2;
        d.P2 = d.n2 * (d.n2 - 1) / 2;
        d.s0 = str_of(X, fp[0]);
        d.s1 = str_of(X, fp[1]);
        d.s2 = str_of(X, kp[0]);
        d.s3 = str_of(X, kp[1]);
        d.scale = 1.0;
        d.row0 = 0;
        d.rows = d.P1;
        d.pbase = 0;
        if (plan.tensors[X.tensor].kind == TKind::INTEGRAL) {
            st.static_src = true;
            plan.tensors[id].static_data = true;
        }
        st.note = "pack " + plan.tensors[X.tensor].name;
        plan.steps.push_back(st);
        return id;
    }

    // out = alpha sum_{k1 k2} A(a1 a2 k1 k2) B(b1 b2 k1 k2) (+ beta out) with A
    // antisymmetric in (a1 a2), (k1 k2) and B in (b1 b2), (k1 k2), as declared:
    // the k-sum runs over k1 < k2 (factor 2) and only a1 < a2, b1 < b2 are
    // computed; the output is filled from them by antisymmetry.
    bool plan_packed(const Stmt &s, const std::vector<char> &lsp, int si, const View &out, BufRef outref,
                     const std::vector<View> &in, double alpha, double beta) {
        if (cplx) { err = "packed index pairs are implemented for real tensors"; return false; }
        const Ref &ra = s.rhs[0], &rb = s.rhs[1];
        std::set<int> Ls(s.rhs[1].letters.begin(), s.rhs[1].letters.end());
        int ka = -1, kb = -1;
        for (int q = 0; q < 2; q++) {
            auto pa = pair_letters(ra, q), pb = pair_letters(rb, q);
            if (Ls.count(pa[0]) && Ls.count(pa[1])) ka = q;
            std::set<int> La(ra.letters.begin(), ra.letters.end());
            if (La.count(pb[0]) && La.count(pb[1])) kb = q;
        }
        if (ka < 0 || kb < 0) { err = "packed pairs: the contracted indices must form a declared pair in both operands"; return false; }
        const auto kpair = pair_letters(ra, ka);               // contracted pair, A's orientation
        const auto fa = pair_letters(ra, 1 - ka), fb = pair_letters(rb, 1 - kb);
        for (const auto &pr : {kpair, fa, fb})
            if (lsp[pr[0]] != lsp[pr[1]]) { err = "a declared pair mixes occupied and virtual indices"; return false; }
        auto up = [](char c) { return c == 'o' ? 'O' : 'V'; };
        std::vector<char> lsp2 = lsp;
        const int LP = (int)lsp2.size(), LQ = LP + 1, LK = LP + 2;
        lsp2.push_back(up(lsp[fa[0]]));
        lsp2.push_back(up(lsp[fb[0]]));
        lsp2.push_back(up(lsp[kpair[0]]));
        const std::string tag = std::to_string(si);
        const int tA = pack_operand(in[0], fa, kpair, lsp2[LP], lsp2[LK], "%pa" + tag, si);
        const int tB = pack_operand(in[1], fb, kpair, lsp2[LQ], lsp2[LK], "%pb" + tag, si);
        if (!err.empty()) return false;
        // C[Q][P] = 2 alpha sum_K Ap[P][K] Bp[Q][K]: an ordinary dense contraction
        Stmt g;
        g.line = s.line;
        g.op = 0;
        g.factor = 2.0 * alpha;
        g.out = Ref{"%pc" + tag, {LQ, LP}, {}};
        g.rhs = {Ref{plan.tensors[tA].name, {LP, LK}, {}}, Ref{plan.tensors[tB].name, {LQ, LK}, {}}};
        if (!plan_stmt(g, lsp2, si)) return false;
        const int tC = last_out;
        version[tC]++;
        last_out = out.tensor;
        // unpack into the output
        Step u;
        u.kind = StepKind::UNPACK;
        u.stmt = si;
        u.a = tensor_ref(tC);
        u.out = outref;
        UnpackDesc &d = u.up;
        if (out.idx.size() != 4) { err = "packed pairs: the output needs four indices"; return false; }
        for (int k = 0; k < 4; k++) {
            d.ext[k] = out.ext[k];
            d.ostr[k] = out.str[k];
        }
        auto pos = [&](int l) {
            for (int k = 0; k < 4; k++)
                if (out.idx[k] == l) return k;
            return -1;
        };
        d.da1 = pos(fa[0]);
        d.da2 = pos(fa[1]);
        d.db1 = pos(fb[0]);
        d.db2 = pos(fb[1]);
        d.nA = ext_of(in[0], fa[0]);
        d.nB = ext_of(in[1], fb[0]);
        d.cA = 1;                                   // C[Q][P]: P fastest
        d.cB = d.nA * (d.nA - 1) / 2;
        d.alpha = 1.0;
        d.beta = beta;
        u.note = "unpack -> " + plan.tensors[out.tensor].name;
        plan.steps.push_back(u);
        return true;
    }

    // K concatenation: the statements ms (binary, no permutation operators, all
    // accumulating into one intermediate, the output's letters split between
    // their operands at the same positions) as one pass over the output placed
    // at the last of them:
    //   C(m, n) += sum_s alpha_s sum_{k in K_s} A_s(m, k) B_s(k, n).
    // Members that contract the same view of the same larger operand (output
    // letters at the same output positions) first have their other operands
    // summed, A B_1 + A B_2 = A (B_1 + B_2), so that operand is read once.  The
    // result runs on the narrow kernel (FP32 plans, one short free side, the
    // members' Y blocks fitting shared memory) or as one split-route GEMM whose
    // planes hold each member's K columns side by side.
    struct KEff {
        View a, b;                  // operands (a holds the output's innermost letter)
        BufRef ar, br;
        double alpha = 1.0;
        std::vector<int> mem;       // members (indices into the group)
        std::set<int> K;            // contracted letters (of the first member)
        int summed = -1;            // 0 / 1: a / b is the sum of the members' operands
        int first = 0;              // the member whose letters the view uses
        std::vector<View> parts;    // summed: each member's operand, relabelled
        std::vector<double> palpha;
    };

    bool plan_kcat(const std::vector<const Stmt *> &ms, const std::vector<const std::vector<char> *> &lsps,
                   const std::vector<int> &sis) {
        const int nm = (int)ms.size();
        std::vector<View> outs(nm), As(nm), Bs(nm);
        std::vector<std::set<int>> Ks(nm);
        std::vector<double> alphas(nm);
        for (int i = 0; i < nm; i++) {
            const Stmt &s = *ms[i];
            if (!resolve(s.out, true, s.op, *lsps[i], outs[i])) return false;
            View in[2];
            for (int k = 0; k < 2; k++)
                if (!resolve(s.rhs[k], false, 0, *lsps[i], in[k])) return false;
            // A holds the output's innermost letter (the GEMM rows; epilogue stores coalesce)
            const int inner = s.out.letters.back();
            std::set<int> L0(s.rhs[0].letters.begin(), s.rhs[0].letters.end());
            const int ia = L0.count(inner) ? 0 : 1;
            As[i] = in[ia];
            Bs[i] = in[1 - ia];
            std::set<int> LA(s.rhs[ia].letters.begin(), s.rhs[ia].letters.end());
            for (int l : s.rhs[1 - ia].letters)
                if (LA.count(l)) Ks[i].insert(l);
            alphas[i] = s.factor * (s.op == -1 ? -1.0 : 1.0) * in[0].sign * in[1].sign;
            last_out = outs[i].tensor;
        }
        const View &out0 = outs[0];
        const Tensor T = plan.tensors[out0.tensor];
        auto pos_of = [&](int i, int letter) {
            const auto &L = ms[i]->out.letters;
            for (size_t p = 0; p < L.size(); p++)
                if (L[p] == letter) return (int)p;
            return -1;
        };
        // the output positions of the rows (A side) and columns (B side), in the
        // output's stride order, from the first member
        auto positions = [&](int i, const View &X) {
            std::set<int> F;
            for (int l : ms[i]->out.letters)
                for (int q : X.idx)
                    if (q == l) F.insert(l);
            return F;
        };
        const std::vector<int> fa0 = fusable(out0, positions(0, As[0])).order;
        const std::vector<int> fb0 = fusable(out0, positions(0, Bs[0])).order;
        std::vector<int> pa, pb;           // output positions of fa0 / fb0
        for (int l : fa0) pa.push_back(pos_of(0, l));
        for (int l : fb0) pb.push_back(pos_of(0, l));
        int64_t Mr = 1, Nr = 1;
        for (int l : fa0) Mr *= ext_of(As[0], l);
        for (int l : fb0) Nr *= ext_of(Bs[0], l);

        // ---- shared operands: member j folds into an earlier member i when its
        // operand on side sd is the same view (output letters at the same output
        // positions, contracted letters where i has contracted ones) of a tensor
        // at least 4x the other operand; mp relabels j's letters as i's
        auto shares = [&](int i, int j, int sd, std::map<int, int> &mp) {
            const View &Xi = sd == 0 ? As[i] : Bs[i], &Xj = sd == 0 ? As[j] : Bs[j];
            const View &Yi = sd == 0 ? Bs[i] : As[i], &Yj = sd == 0 ? Bs[j] : As[j];
            if (Xi.tensor != Xj.tensor || Xi.idx.size() != Xj.idx.size()) return false;
            if (view_elems(Xi) < 4 * view_elems(Yi) || view_elems(Xj) < 4 * view_elems(Yj)) return false;
            mp.clear();
            for (size_t d = 0; d < Xi.idx.size(); d++) {
                const int li = Xi.idx[d], lj = Xj.idx[d];
                const int p_i = pos_of(i, li), p_j = pos_of(j, lj);
                if ((p_i < 0) != (p_j < 0) || p_i != p_j) return false;
                mp[lj] = li;
            }
            std::set<int> got, want(Yi.idx.begin(), Yi.idx.end());
            for (int l : Yj.idx) {
                const int p_j = pos_of(j, l);
                if (p_j >= 0) mp[l] = ms[i]->out.letters[p_j];
                else if (!mp.count(l)) return false;
                got.insert(mp[l]);
            }
            return got == want && got.size() == Yj.idx.size();
        };
        std::vector<int> rep(nm, -1), rep_side(nm, -1);
        std::vector<std::map<int, int>> relabel(nm);
        for (int j = 1; j < nm; j++)
            for (int i = 0; i < j && rep[j] < 0; i++) {
                if (rep[i] >= 0) continue;
                for (int sd = 0; sd < 2 && rep[j] < 0; sd++) {
                    if (rep_side[i] >= 0 && rep_side[i] != sd) continue;
                    std::map<int, int> mp;
                    if (shares(i, j, sd, mp)) {
                        rep[j] = i;
                        rep_side[i] = sd;
                        relabel[j] = mp;
                    }
                }
            }
        std::vector<KEff> eff;
        for (int i = 0; i < nm; i++) {
            if (rep[i] >= 0) continue;
            KEff e;
            e.a = As[i];
            e.b = Bs[i];
            e.ar = tensor_ref(As[i].tensor);
            e.br = tensor_ref(Bs[i].tensor);
            e.alpha = alphas[i];
            e.K = Ks[i];
            e.first = i;
            e.mem.push_back(i);
            for (int j = i + 1; j < nm; j++)
                if (rep[j] == i) e.mem.push_back(j);
            if (e.mem.size() > 1) {
                const int sd = rep_side[i];
                e.summed = 1 - sd;
                for (int j : e.mem) {
                    View y = sd == 0 ? Bs[j] : As[j];
                    if (j != i)
                        for (int &l : y.idx) l = relabel[j][l];
                    e.parts.push_back(y);
                    e.palpha.push_back(alphas[j]);
                }
                const View &y0 = sd == 0 ? Bs[i] : As[i];
                View w = contiguous_view(y0.idx, y0);
                (sd == 0 ? e.b : e.a) = w;
                e.alpha = 1.0;
            }
            eff.push_back(e);
        }
        const int ne = (int)eff.size();
        std::vector<int64_t> kx(ne), slot(ne);
        int64_t ktot = 0;
        for (int i = 0; i < ne; i++) {
            kx[i] = 1;
            for (int l : eff[i].K) kx[i] *= ext_of(eff[i].a, l);
            slot[i] = align_up(kx[i], 8);
            ktot += slot[i];
        }
        // the members' letters for the first member's row / column / output orders
        auto mapped = [&](const KEff &e, const std::vector<int> &ps) {
            std::vector<int> r;
            for (int p : ps) r.push_back(ms[e.first]->out.letters[p]);
            return r;
        };
        auto sum_steps = [&](KEff &e, int si) {
            // the summed operand: a contiguous scratch buffer in the first member's layout
            View &w = e.summed == 0 ? e.a : e.b;
            BufRef &wr = e.summed == 0 ? e.ar : e.br;
            wr = scratch(view_elems(w) * esz);
            for (size_t q = 0; q < e.parts.size(); q++) {
                const int j = e.mem[q];
                const View &src = e.parts[q];
                Step st = accum_step(w, wr, src, tensor_ref(src.tensor), std::vector<Perm>(1, Perm{1.0, {}}),
                                     e.palpha[q], q == 0 ? 0.0 : 1.0);
                if (!err.empty()) return false;
                st.stmt = si;
                st.note = std::string(q == 0 ? "operand sum = " : "operand sum += ") + plan.tensors[src.tensor].name +
                          " (statement " + std::to_string(sis[j] + 1) + ")";
                plan.steps.push_back(st);
            }
            return true;
        };
        std::string note = "K-concatenated:";
        for (int i = 0; i < ne; i++) {
            note += i ? " + " : " ";
            const KEff &e = eff[i];
            auto nm_of = [&](int sd) {
                if (e.summed != sd) return plan.tensors[(sd == 0 ? e.a : e.b).tensor].name;
                std::string x = "(";
                for (size_t q = 0; q < e.parts.size(); q++) x += (q ? "+" : "") + plan.tensors[e.parts[q].tensor].name;
                return x + ")";
            };
            note += nm_of(0) + "*" + nm_of(1);
        }
        note += " -> " + T.name;

        // ---- the narrow kernel: FP32 plans, one free side of at most 64, the long
        // side in 32-bit range, every member's Y block in shared memory
        const bool xa = Mr >= Nr;
        const int64_t R = xa ? Mr : Nr, NCx = xa ? Nr : Mr;
        if (plan.precision == 2 && !cplx && ne <= kMaxRowsMembers && NCx >= 1 && NCx <= 64 && R >= 4096 &&
            R <= 0xffffffffLL) {
            RowsMultiDesc d{};
            d.R = R;
            d.nc = (int)NCx;
            d.nm = ne;
            d.f32 = 1;
            for (int i = 0; i < ne; i++) d.m[i].K = (int)kx[i];
            if (rows_multi_smem_bytes(d) > 0 && rows_multi_smem_bytes(d) <= 96 * 1024) {
                scratch_need = 0;
                for (auto &e : eff)
                    if (e.summed >= 0 && !sum_steps(e, sis.back())) return false;
                Step g;
                g.kind = StepKind::GEMM;
                g.stmt = sis.back();
                g.rows = true;
                g.kstmts = sis;
                g.gemm.M = Mr;
                g.gemm.N = Nr;
                g.gemm.K = 0;
                g.gemm.splitk = 1;
                g.gemm.f32 = 1;
                const View &X0 = xa ? eff[0].a : eff[0].b, &Y0 = xa ? eff[0].b : eff[0].a;
                d.cr = make_grp(mapped(eff[0], xa ? pa : pb), X0, outs[eff[0].first]);
                d.cc = make_grp(mapped(eff[0], xa ? pb : pa), Y0, outs[eff[0].first]);
                for (int i = 0; i < ne; i++) {
                    const KEff &e = eff[i];
                    const View &X = xa ? e.a : e.b, &Y = xa ? e.b : e.a;
                    const std::vector<int> rord = mapped(e, xa ? pa : pb), cord = mapped(e, xa ? pb : pa);
                    const std::vector<int> kord = fusable(X, e.K).order;
                    RowsMember &m = d.m[i];
                    m.xr = make_grp(rord, X, X);
                    m.xk = make_grp(kord, X, X);
                    m.yk = make_grp(kord, Y, Y);
                    m.yc = make_grp(cord, Y, Y);
                    m.alpha = e.alpha;
                    KMember mb;
                    mb.stmt = sis[e.first];
                    mb.a = xa ? e.ar : e.br;     // X
                    mb.b = xa ? e.br : e.ar;     // Y
                    mb.flops = 2.0 * (double)Mr * (double)Nr * (double)kx[i];
                    g.flops += mb.flops;
                    g.gemm.K += kx[i];
                    g.kcat.push_back(mb);
                }
                if (!err.empty()) return false;
                for (int i = 0; i < nm; i++)
                    if (rep[i] >= 0) {
                        // folded members: their flops as if run on their own
                        int64_t k = 1;
                        for (int l : Ks[i]) k *= ext_of(As[i], l);
                        g.flops += 2.0 * (double)Mr * (double)Nr * (double)k;
                    }
                g.rm = d;
                g.rg.red = 0;
                g.cands = {{0, 1, 0}, {0, 1, 1}};
                g.out = tensor_ref(out0.tensor);
                g.note = note;
                plan.flops += g.flops;
                plan.steps.push_back(g);
                return true;
            }
        }

        // ---- the split route: HBM bytes of the merged GEMM against the members
        // run one by one.  The merge saves a read-modify-write pass over the
        // output per statement and costs the planes of the whole padded K
        // (written by the splits, read by the GEMM).  Alone, a statement takes
        // the split route on the terms of plan_stmt (large, not narrow, tiles
        // filled), and an integral (or integral-only) operand's planes are then
        // cached once per solve, so only their read counts.  Effective members
        // that cost more merged than alone are left out (kcat_keep); the rest
        // merge if they still save bytes.
        const int np = plan.precision == 3 ? 3 : 2;
        {
            const double out_rmw = 16.0 * (double)Mr * (double)Nr;
            const double rows_x[2] = {(double)Mr, (double)Nr};
            double merged = out_rmw + 4.0 * np * (double)(Mr + Nr) * (double)(align_up(ktot, 64) - ktot), alone = 0.0;
            kcat_keep.assign(nm, 1);
            int kept = 0;
            auto alone_bytes = [&](const View &A, const View &B, int64_t K) {
                const View *ops[2] = {&A, &B};
                const bool narrow = K <= 64 && std::min(Mr, Nr) >= 2 && std::min(Mr, Nr) <= 64 && std::max(Mr, Nr) >= 4096;
                const int64_t bn = Nr <= 64 ? 64 : Nr <= 128 ? 128 : 256;
                const double eff_t = (double)Mr * (double)Nr * (double)K /
                                     ((double)align_up(Mr, 128) * (double)align_up(Nr, bn) * (double)align_up(K, 64));
                const bool split = 2.0 * (double)Mr * (double)Nr * (double)K >= 2.0e8 && Mr > 1 && Nr > 1 && K > 1 &&
                                   !(narrow && eff_t < 0.5) && eff_t >= 0.15;
                double a_i = out_rmw;
                for (int x = 0; x < 2; x++) {
                    const double bytes = 8.0 * (double)view_elems(*ops[x]);
                    const double planes = 2.0 * np * rows_x[x] * (double)align_up(K, 64);
                    const Tensor &tx = plan.tensors[ops[x]->tensor];
                    const bool cached = tx.kind == TKind::INTEGRAL || tx.static_data;
                    a_i += !split ? bytes : cached ? planes : bytes + 2.0 * planes;
                }
                return a_i;
            };
            for (int i = 0; i < ne; i++) {
                const KEff &e = eff[i];
                double m_i = 4.0 * np * (double)(Mr + Nr) * (double)slot[i], a_i = 0.0;
                for (int j : e.mem) {
                    int64_t k = 1;
                    for (int l : Ks[j]) k *= ext_of(As[j], l);
                    a_i += alone_bytes(As[j], Bs[j], k);
                    m_i += 8.0 * (double)(view_elems(As[j]) + view_elems(Bs[j]));
                }
                if (e.summed >= 0) {
                    // the shared operand is read once, the summed one written and read
                    const View &sh = e.summed == 0 ? e.b : e.a, &sm = e.summed == 0 ? e.a : e.b;
                    m_i -= 8.0 * (double)view_elems(sh) * (double)(e.mem.size() - 1);
                    m_i += 16.0 * (double)view_elems(sm);
                }
                if (m_i >= a_i) {
                    for (int j : e.mem) kcat_keep[j] = 0;
                    continue;
                }
                kept += (int)e.mem.size();
                merged += m_i;
                alone += a_i;
            }
            if (kept < nm || merged >= alone) {
                if (merged >= alone) kcat_keep.assign(nm, 0);
                kcat_declined = true;
                return true;
            }
        }
        scratch_need = 0;
        for (auto &e : eff)
            if (e.summed >= 0 && !sum_steps(e, sis.back())) return false;
        Step g;
        g.kind = StepKind::GEMM;
        g.stmt = sis.back();
        g.mixed = true;
        g.kstmts = sis;
        TcGemmDesc &t = g.tc;
        t.M = Mr;
        t.N = Nr;
        t.bn = Nr <= 64 ? 64 : (Nr <= 128 || np == 3) ? 128 : 256;
        const int bn_max = np == 3 ? (Nr <= 64 ? 64 : 128) : (Nr <= 64 ? 64 : Nr <= 128 ? 128 : 256);
        t.Mp = align_up(Mr, 128);
        t.Np = align_up(Nr, bn_max);
        t.Kp = align_up(ktot, 64);
        const int64_t tiles = (t.Mp / 128) * ((Nr + t.bn - 1) / t.bn), kblocks = t.Kp / 64;
        t.splitk = 1;
        if (tiles < 148 && kblocks >= 8) {
            int64_t sk = std::min<int64_t>((148 + tiles - 1) / tiles, kblocks / 4);
            if (sk > 1) t.splitk = (int)sk;
        }
        int64_t skmax = t.splitk;
        for (int bn : {64, 128, 256}) {
            if (bn > bn_max) continue;
            for (int sk : {1, 2, 4, 8, 16})
                if (sk == 1 || (sk <= kblocks / 4 && sk * Mr * Nr * 8 <= (int64_t)512 << 20)) {
                    g.cands.push_back({bn, sk, 0});
                    skmax = std::max<int64_t>(skmax, sk);
                }
            g.cands.push_back({bn, 1, 1});       // accumulating: the reduction epilogue
        }
        const std::array<int, 3> planned{t.bn, t.splitk, 0};
        if (std::find(g.cands.begin(), g.cands.end(), planned) == g.cands.end()) g.cands.push_back(planned);
        if (skmax > 1) g.partials = scratch(skmax * Mr * Nr * 8);
        t.nplanes_a = t.nplanes_b = np;
        if (np == 2) {
            const int pa_[3] = {0, 0, 1}, pb_[3] = {0, 1, 0};
            t.nprod = 3;
            for (int k = 0; k < 3; k++) { t.prod_a[k] = pa_[k]; t.prod_b[k] = pb_[k]; }
        } else {
            const int pa_[6] = {0, 0, 1, 0, 1, 2}, pb_[6] = {0, 1, 0, 2, 1, 0};
            t.nprod = 6;
            for (int k = 0; k < 6; k++) { t.prod_a[k] = pa_[k]; t.prod_b[k] = pb_[k]; }
        }
        t.cm = make_grp(fa0, As[0], out0);
        t.cn = make_grp(fb0, Bs[0], out0);
        t.alpha = 1.0;                            // each member's factor rides on its A split
        t.beta = 1.0;
        g.out = tensor_ref(out0.tensor);
        int64_t koff = 0;
        for (int i = 0; i < ne; i++) {
            const KEff &e = eff[i];
            KMember mb;
            mb.stmt = sis[e.first];
            mb.a = e.ar;
            mb.b = e.br;
            const std::vector<int> fa = mapped(e, pa), fb = mapped(e, pb);
            const View &big = view_elems(e.a) >= view_elems(e.b) ? e.a : e.b;
            const std::vector<int> korder = fusable(big, e.K).order;
            const int64_t kend = i == ne - 1 ? t.Kp - koff : slot[i];
            SplitDesc &sa = mb.split_a;
            sa.R = Mr; sa.K = kx[i]; sa.Rp = Mr; sa.Kp = t.Kp; sa.nplanes = np;
            sa.gr = make_grp(fa, e.a, e.a);
            sa.gk = make_grp(korder, e.a, e.a);
            sa.kdst = koff; sa.kend = kend;
            sa.scaled = e.alpha != 1.0;
            sa.scale = e.alpha;
            SplitDesc &sb = mb.split_b;
            sb.R = Nr; sb.K = kx[i]; sb.Rp = Nr; sb.Kp = t.Kp; sb.nplanes = np;
            sb.gr = make_grp(fb, e.b, e.b);
            sb.gk = make_grp(korder, e.b, e.b);
            sb.kdst = koff; sb.kend = kend;
            if (!err.empty()) return false;
            mb.flops = 2.0 * (double)Mr * (double)Nr * (double)kx[i];
            koff += slot[i];
            g.kcat.push_back(mb);
        }
        for (int i = 0; i < nm; i++) {
            int64_t k = 1;
            for (int l : Ks[i]) k *= ext_of(As[i], l);
            g.flops += 2.0 * (double)Mr * (double)Nr * (double)k;
        }
        g.note = note;
        // the merged planes are read by this step only: they live in the
        // statement arena (rebased after planning), shared with every other step
        g.planes_a_off = scratch(planes_bytes(Mr, t.Kp, np)).off;
        g.planes_b_off = scratch(planes_bytes(Nr, t.Kp, np)).off;
        plan.flops += g.flops;
        plan.flops_mixed += g.flops;
        plan.steps.push_back(g);
        return true;
    }

    bool plan_stmt(const Stmt &s, const std::vector<char> &lsp, int si) {
        View out;
        if (!resolve(s.out, true, s.op, lsp, out)) return false;
        last_out = out.tensor;
        const Tensor T = plan.tensors[out.tensor];
        if (T.kind != TKind::RES && T.kind != TKind::INTERM) { err = "output must be a residual or an intermediate"; return false; }
        std::vector<View> in(s.rhs.size());
        for (size_t k = 0; k < s.rhs.size(); k++)
            if (!resolve(s.rhs[k], false, 0, lsp, in[k])) return false;
        for (auto &w : in)
            if (w.tensor == out.tensor) { err = "output also used as an operand"; return false; }
        std::set<int> O(s.out.letters.begin(), s.out.letters.end());
        for (auto &pp : s.perms) {
            for (int l : pp.first)
                if (!O.count(l)) { err = "permutation index not in the output"; return false; }
            for (int l : pp.first)
                if (lsp[l] != lsp[pp.first[0]]) { err = "permutation mixes occupied and virtual indices"; return false; }
        }
        std::vector<Perm> perms = expand_perms(s.perms);
        double alpha = s.factor * (s.op == -1 ? -1.0 : 1.0);
        for (auto &w : in) {
            alpha *= w.sign;
            if (w.conj && plan.dtype == 0) w.conj = false;   // real integrals: bra<->ket symmetric
        }
        double beta = s.op == 0 ? 0.0 : 1.0;
        BufRef outref = tensor_ref(out.tensor);
        if (!initialized[out.tensor] && s.op != 0) {
            if (T.kind == TKind::INTERM) { err = "intermediate accumulated before it is defined"; return false; }
            // the first accumulation into a residual assigns it (every route
            // writes every element of its output): no zeroing pass
            beta = 0.0;
        }
        initialized[out.tensor] = true;

        if (in.size() == 1) {
            std::set<int> A(s.rhs[0].letters.begin(), s.rhs[0].letters.end());
            if (A != O) { err = "a single-tensor statement must carry exactly the output's indices"; return false; }
            Step st = accum_step(out, outref, in[0], tensor_ref(in[0].tensor), perms, alpha, beta);
            if (!err.empty()) return false;
            st.stmt = si;
            st.note = "copy " + plan.tensors[in[0].tensor].name + " -> " + T.name;
            plan.steps.push_back(st);
            return true;
        }

        // binary contraction
        std::set<int> LA(s.rhs[0].letters.begin(), s.rhs[0].letters.end());
        std::set<int> LB(s.rhs[1].letters.begin(), s.rhs[1].letters.end());
        std::set<int> K, FA, FB;
        for (int l : LA) (LB.count(l) ? K : FA).insert(l);
        for (int l : LB)
            if (!LA.count(l)) FB.insert(l);
        for (int l : K)
            if (O.count(l)) { err = "an index in both operands and in the output (Hadamard product) is not supported"; return false; }
        std::set<int> F;
        F.insert(FA.begin(), FA.end());
        F.insert(FB.begin(), FB.end());
        if (F != O) { err = "output indices must be exactly the uncontracted operand indices"; return false; }

        // packed pairs: each operand is two declared antisymmetric pairs, one of
        // them contracted (e.g. the particle ladder tau[(ij)(ef)] * V[(ab)(ef)])
        if (s.rhs[0].pairs.size() == 2 && s.rhs[1].pairs.size() == 2 && s.rhs[0].letters.size() == 4 &&
            s.rhs[1].letters.size() == 4 && K.size() == 2 && perms.size() == 1 && perms[0].sigma.empty())
            return plan_packed(s, lsp, si, out, outref, in, alpha, beta);

        if (K.empty()) {
            // outer product: each output element is formed directly as a sum of
            // signed products (no GEMM, no scratch, no separate antisymmetrisation)
            Step st = accum_step(out, outref, in[0], tensor_ref(in[0].tensor), perms, alpha, beta);
            if (!err.empty()) return false;
            st.acc.two_src = 1;
            for (int p = 0; p < st.acc.nperm; p++)
                for (int k = 0; k < st.acc.nd; k++) {
                    int mu = out.idx[k], pre = mu;
                    for (auto &kv : perms[p].sigma)
                        if (kv.second == mu) pre = kv.first;
                    st.acc.sstr[p][k] = str_of(in[0], pre);
                    st.acc.sstr2[p][k] = str_of(in[1], pre);
                }
            st.b = tensor_ref(in[1].tensor);
            st.acc.conj_b = cplx && in[1].conj ? 1 : 0;
            st.stmt = si;
            st.note = "outer " + plan.tensors[in[0].tensor].name + "*" + plan.tensors[in[1].tensor].name + " -> " + T.name;
            plan.steps.push_back(st);
            return true;
        }

        // GEMM rows (A side) get the operand whose free indices hold the
        // output's fastest index, so epilogue stores coalesce along rows.
        int ia = 0, ib = 1;
        {
            int inner = out.idx.back();
            if (FB.count(inner)) { std::swap(ia, ib); std::swap(FA, FB); }
        }
        View A = in[ia], B = in[ib];
        BufRef aref = tensor_ref(A.tensor), bref = tensor_ref(B.tensor);
        int64_t Mx = 1, Nx = 1, Kx = 1;
        for (int l : FA) Mx *= ext_of(A, l);
        for (int l : FB) Nx *= ext_of(B, l);
        for (int l : K) Kx *= ext_of(A, l);
        // real flops: a complex multiply-add is four real ones
        const double flops = (cplx ? 8.0 : 2.0) * (double)Mx * (double)Nx * (double)Kx;
        scratch_need = 0;
        // split-bf16 route: contractions of >= 2e8 flops that are real GEMMs
        // (matrix-vector shapes stay on the memory-bound FP64 kernels)
        bool use_mixed = plan.precision != 0 &&
                         (mixed_all || (flops >= 2.0e8 && Mx > 1 && Nx > 1 && Kx > 1));
        // exact-slice plans (FP64-grade): every other route stays FP64
        const bool slices = plan.precision == 4;
        // except a matrix-vector product against a large integral block: its
        // split planes are cached once per solve, so the tensor route streams
        // half the bytes of the FP64 block (the idle tile columns cost nothing
        // next to that)
        const auto big_static = [&](const View &X) {
            return plan.tensors[X.tensor].kind == TKind::INTEGRAL && view_elems(X) >= 100000000;
        };
        const bool static_mv = plan.precision != 0 && !slices && !mixed_all && Kx > 1 && (Mx == 1) != (Nx == 1) &&
                               (big_static(A) || big_static(B));
        use_mixed = use_mixed || static_mv;
        // Tensor tiles are 128 x bn x 64.  A narrow contraction (K <= 64 and one
        // free side <= 64, e.g. the rank-o updates of T3) that fills them less
        // than half is memory-bound: it runs on the narrow kernel with FP32
        // arithmetic.  Anything else stays on the tensor cores unless they
        // would waste more than ~85% of the tile (then: FP32 SIMT GEMM).
        const bool narrow = !cplx && Kx >= 2 && Kx <= 64 && std::min(Mx, Nx) >= 2 && std::min(Mx, Nx) <= 64 &&
                            std::max(Mx, Nx) >= 4096 && std::max(Mx, Nx) <= 0xffffffffLL;
        bool use_f32 = false;
        bool use_rows = narrow;
        // bf16x3 plans carry ~2^-16 relative error on their bulk contractions:
        // the contractions below the tensor-route size run in FP32 arithmetic
        // there (the SIMT FP32 rate, ~60x the FP64 pipe); bf16x6 and FP64 plans
        // keep FP64 for them
        if (!use_mixed && !mixed_all && plan.precision == 2 && !cplx && Mx > 1 && Nx > 1 && Kx > 1) use_f32 = true;
        // uniform plans (the same steps at any size): a contraction with a
        // two-index operand (T1 or an F intermediate) goes to the narrow kernel,
        // every other one to the split route, whatever the extents
        if (uniform) {
            const bool mat = s.rhs[0].letters.size() == 2 || s.rhs[1].letters.size() == 2;
            use_mixed = !mat;
            use_rows = mat;
            use_f32 = mat && plan.precision == 2;
        }
        if (use_mixed && !mixed_all) {
            const int64_t bn = Nx <= 64 ? 64 : Nx <= 128 ? 128 : 256;
            const double eff = (double)Mx * (double)Nx * (double)Kx /
                               ((double)align_up(Mx, 128) * (double)align_up(Nx, bn) * (double)align_up(Kx, 64));
            if (narrow && eff < 0.5) {
                use_mixed = false;
                use_rows = true;
                use_f32 = !slices;
            } else if (eff < 0.15 && !cplx && !static_mv) {
                use_mixed = false;
                use_f32 = !slices;
            }
        }

        // A long contraction with at most 8 columns on the small operand's side
        // (the reductions of T3 against integrals and small intermediates): the
        // large operand is read in place by the narrow_k kernel when its
        // contraction ends in a unit-stride run of at least 32 that the other
        // operand also holds as one strided run; no permuted copy is made.
        const bool x_is_a = view_elems(A) >= view_elems(B);
        const View &Xn = x_is_a ? A : B, &Yn = x_is_a ? B : A;
        const int64_t n_free = x_is_a ? Nx : Mx, m_free = x_is_a ? Mx : Nx;
        std::vector<int> nk_outer;
        int64_t nk_L = 1, nk_sy = 0;
        bool use_nk = false;
        if (!cplx && !use_mixed && !use_rows && n_free <= 8 && Kx >= 256 && view_elems(Xn) >= ((int64_t)1 << 20) &&
            plan.tensors[Yn.tensor].elems < ((int64_t)1 << 31)) {
            std::vector<int> kl;
            for (int l : fusable(Xn, K).order)
                if (ext_of(Xn, l) > 1) kl.push_back(l);
            size_t cut = kl.size();
            int64_t ex = 1, ey = 0;
            while (cut > 0) {
                const int l = kl[cut - 1];
                const int64_t sx = str_of(Xn, l), sy = str_of(Yn, l), e = ext_of(Xn, l);
                if (sx != ex || (cut < kl.size() && sy != ey)) break;
                if (cut == kl.size()) nk_sy = sy;
                ex = sx * e;
                ey = sy * e;
                nk_L *= e;
                cut--;
            }
            nk_outer.assign(kl.begin(), kl.begin() + cut);
            use_nk = nk_L >= 32 && m_free >= 1;
        }

        Step g;
        g.kind = StepKind::GEMM;
        g.stmt = si;
        g.flops = flops;
        g.note = plan.tensors[A.tensor].name + "*" + plan.tensors[B.tensor].name + " -> " + T.name;
        std::vector<int> fa_order, fb_order, k_order;

        // narrow contractions (short K, one short free side): one thread per
        // row of the long side, every operand read in place through its strides
        if (use_rows && !use_mixed) {
            const bool direct0 = perms.size() == 1 && perms[0].sigma.empty();
            fa_order = direct0 ? fusable(out, FA).order : fusable(A, FA).order;
            fb_order = direct0 ? fusable(out, FB).order : fusable(B, FB).order;
            k_order = Mx >= Nx ? fusable(A, K).order : fusable(B, K).order;
            g.rows = true;
            g.gemm.splitk = 1;
            g.gemm.M = Mx;
            g.gemm.N = Nx;
            g.gemm.K = Kx;
            g.gemm.f32 = use_f32 ? 1 : 0;
        } else if (use_nk) {
            std::set<int> FX = x_is_a ? FA : FB, FY = x_is_a ? FB : FA;
            (x_is_a ? fa_order : fb_order) = fusable(Xn, FX).order;
            (x_is_a ? fb_order : fa_order) = fusable(Yn, FY).order;
            g.nk = true;
            g.gemm.splitk = 1;
            g.gemm.M = m_free;
            g.gemm.N = n_free;
            g.gemm.K = Kx;
            // bf16x3 plans: FP32 products here too, matrix-vector shapes included
            // (their FP32 accumulation error sits far below the split route's
            // 2^-16; in FP64 the narrow FP64 pipe bounds them)
            g.gemm.f32 = (use_f32 || (plan.precision == 2 && !cplx)) ? 1 : 0;
        } else if (use_mixed) {
            // The split kernels read any strided view: no permutes on this route,
            // and the row/column orders are free.  Rows and columns follow the
            // output's stride order (consecutive rows -> the output's fastest
            // index, so epilogue stores coalesce); K follows the larger operand.
            if (perms.size() == 1 && perms[0].sigma.empty()) {
                fa_order = fusable(out, FA).order;
                fb_order = fusable(out, FB).order;
            } else {
                fa_order = fusable(A, FA).order;
                fb_order = fusable(B, FB).order;
            }
            k_order = view_elems(A) >= view_elems(B) ? fusable(A, K).order : fusable(B, K).order;
            g.mixed = true;
        } else {
            Fuse fa = fusable(A, FA), ka = fusable(A, K), fb = fusable(B, FB), kb = fusable(B, K);
            bool a_ok = fa.ok && ka.ok, b_ok = fb.ok && kb.ok;
            bool match = a_ok && b_ok && same_order(A, ka.order, B, kb.order);
            bool perm_a = false, perm_b = false;
            std::vector<int> korder = ka.order;
            if (!match) {
                if (a_ok && (!b_ok || view_elems(B) <= view_elems(A))) { perm_b = true; korder = ka.order; }
                else if (b_ok) { perm_a = true; korder = kb.order; }
                else { perm_a = perm_b = true; korder = ka.order; }
            }
            auto do_perm = [&](View &X, BufRef &xref, const std::vector<int> &forder) {
                std::vector<int> ord = forder;
                ord.insert(ord.end(), korder.begin(), korder.end());
                View w = contiguous_view(ord, X);
                // an integral block's permuted copy is static: it lives in the cache region
                // and is rebuilt only when the cache is invalid (every cc_residual call,
                // once per cc_solve)
                const bool stat = plan.tensors[X.tensor].kind == TKind::INTEGRAL;
                BufRef r;
                if (stat) {
                    r.where = BufRef::WS;
                    r.slot = 2;                 // cache-relative, rebased after planning
                    r.off = cache_need;
                    cache_need += align_up(view_elems(w) * esz);
                } else {
                    r = scratch(view_elems(w) * esz);
                }
                Step p = accum_step(w, r, X, xref, std::vector<Perm>(1, Perm{1.0, {}}), 1.0, 0.0);
                if (!err.empty()) return;
                p.static_src = stat;
                p.stmt = si;
                p.note = std::string(stat ? "permute (cached) " : "permute ") + plan.tensors[X.tensor].name;
                plan.steps.push_back(p);
                w.tensor = X.tensor;
                w.sign = X.sign;
                w.conj = false;             // applied by the permute
                X = w;
                xref = r;
            };
            if (perm_a) do_perm(A, aref, fa.order);
            if (perm_b) do_perm(B, bref, fb.order);
            if (!err.empty()) return false;
            Fuse fa2 = fusable(A, FA), ka2 = fusable(A, K), fb2 = fusable(B, FB), kb2 = fusable(B, K);
            if (!(fa2.ok && ka2.ok && fb2.ok && kb2.ok && same_order(A, ka2.order, B, kb2.order))) {
                err = "internal: operands not GEMM-ready after permutes";
                return false;
            }
            fa_order = fa2.order;
            fb_order = fb2.order;
            k_order = ka2.order;
            g.gemm.M = fa2.extent;
            g.gemm.N = fb2.extent;
            g.gemm.K = ka2.extent;
            g.gemm.sAm = g.gemm.M == 1 ? 1 : fa2.stride;
            g.gemm.sAk = g.gemm.K == 1 ? 1 : ka2.stride;
            g.gemm.sBk = g.gemm.K == 1 ? 1 : kb2.stride;
            g.gemm.sBn = g.gemm.N == 1 ? 1 : fb2.stride;
            if (!(g.gemm.sAm == 1 || g.gemm.sAk == 1) || !(g.gemm.sBk == 1 || g.gemm.sBn == 1)) {
                err = "internal: GEMM operand without a unit stride";
                return false;
            }
            // split K when the output has too few 64x64 tiles to fill the SMs
            const int64_t tiles = ((g.gemm.M + 63) / 64) * ((g.gemm.N + 63) / 64);
            g.gemm.splitk = 1;
            if (tiles < 296 && g.gemm.K >= 512 && g.gemm.M > 1 && g.gemm.N > 1) {
                int64_t sk = (592 + tiles - 1) / tiles;
                sk = std::min<int64_t>(sk, g.gemm.K / 128);
                sk = std::min<int64_t>(sk, 256);
                if (sk > 1) g.gemm.splitk = (int)sk;
            }
            // autotuning candidates: split-K factors (the partials buffer takes the largest)
            int64_t skmax = g.gemm.splitk;
            if (g.gemm.M > 1 && g.gemm.N > 1 && g.gemm.K > 1) {
                g.cands.push_back({0, 1, 0});
                for (int sk : {2, 4, 8, 16, 32, 64})
                    if (sk <= g.gemm.K / 64 && sk * g.gemm.M * g.gemm.N * esz <= (int64_t)512 << 20) {
                        g.cands.push_back({0, sk, 0});
                        skmax = std::max<int64_t>(skmax, sk);
                    }
                if (g.gemm.splitk > 1 &&
                    std::find(g.cands.begin(), g.cands.end(), std::array<int, 3>{0, g.gemm.splitk, 0}) == g.cands.end())
                    g.cands.push_back({0, g.gemm.splitk, 0});
                if (g.cands.size() < 2) g.cands.clear();
            }
            if (skmax > 1) g.partials = scratch(skmax * g.gemm.M * g.gemm.N * esz);
        }

        // output: direct (generalised strides) or scratch + antisymmetrising epilogue
        const bool direct = perms.size() == 1 && perms[0].sigma.empty();
        View Cv;
        BufRef cref;
        double galpha = alpha, gbeta = beta;
        if (direct) {
            Cv = out;
            cref = outref;
        } else {
            // scratch [FB][FA]: the GEMM's row index (A side) is the fastest
            std::vector<int> ord = fb_order;
            ord.insert(ord.end(), fa_order.begin(), fa_order.end());
            Cv = contiguous_view(ord, A, &B);
            cref = scratch(view_elems(Cv) * esz);
            gbeta = 0.0;
        }
        Grp cm = make_grp(fa_order, A, Cv), cn = make_grp(fb_order, B, Cv);
        if (!err.empty()) return false;
        g.out = cref;
        g.a = aref;
        g.b = bref;
        if (g.nk) {
            NarrowKDesc &d = g.nkd;
            const std::vector<int> &rord = x_is_a ? fa_order : fb_order, &cord = x_is_a ? fb_order : fa_order;
            d.M = m_free;
            d.N = (int)n_free;
            d.L = nk_L;
            d.sy = nk_sy;
            d.Ko = 1;
            for (int l : nk_outer) d.Ko *= ext_of(Xn, l);
            d.xm = make_grp(rord, Xn, Xn);
            d.xko = make_grp(nk_outer, Xn, Xn);
            d.yko = make_grp(nk_outer, Yn, Yn);
            d.yn = make_grp(cord, Yn, Yn);
            d.cm = make_grp(rord, Xn, Cv);
            d.cn = make_grp(cord, Yn, Cv);
            if (!err.empty()) return false;
            d.alpha = galpha;
            d.beta = gbeta;
            d.f32 = g.gemm.f32;                  // as chosen with the route above
            g.gemm.alpha = galpha;
            g.gemm.beta = gbeta;
            g.gemm.cm = cm;
            g.gemm.cn = cn;
            // about 4096 elements of a row per work item (whole runs when they are
            // shorter), but enough items to keep 48 warps on every SM
            const int64_t groups = (d.M + 3) / 4;
            auto items = [&] { return groups * ((d.Ko + d.kper - 1) / d.kper) * ((d.L + d.seg - 1) / d.seg); };
            d.kper = std::max<int64_t>(1, 4096 / d.L);
            d.seg = std::min<int64_t>(d.L, 4096);
            while (d.kper > 1 && items() < 148 * 48) d.kper /= 2;
            while (d.kper == 1 && d.seg > 512 && items() < 148 * 48) d.seg = align_up(d.seg / 2, 64);
            g.a = x_is_a ? aref : bref;
            g.b = x_is_a ? bref : aref;
        } else if (g.rows) {
            RowsGemmDesc &r = g.rg;
            const bool xa = Mx >= Nx;
            const View &X = xa ? A : B, &Y = xa ? B : A;
            const std::vector<int> &rord = xa ? fa_order : fb_order, &cord = xa ? fb_order : fa_order;
            r.R = xa ? Mx : Nx;
            r.nc = (int)(xa ? Nx : Mx);
            r.K = (int)Kx;
            r.xr = make_grp(rord, X, X);
            r.xk = make_grp(k_order, X, X);
            r.yk = make_grp(k_order, Y, Y);
            r.yc = make_grp(cord, Y, Y);
            r.cr = make_grp(rord, X, Cv);
            r.cc = make_grp(cord, Y, Cv);
            if (!err.empty()) return false;
            r.alpha = galpha;
            r.beta = gbeta;
            r.f32 = use_f32 ? 1 : 0;
            // an accumulating narrow GEMM may add its outputs with reductions
            if (gbeta == 1.0) g.cands = {{0, 1, 0}, {0, 1, 1}};
            g.a = xa ? aref : bref;
            g.b = xa ? bref : aref;
        } else if (!g.mixed) {
            g.gemm.cm = cm;
            g.gemm.cn = cn;
            g.gemm.alpha = galpha;
            g.gemm.beta = gbeta;
            // an accumulating tiled GEMM may add its outputs with reductions
            if (gbeta == 1.0 && !g.cands.empty()) g.cands.push_back({0, 1, 1});
            g.gemm.f32 = use_f32 ? 1 : 0;
            g.gemm.cplx = cplx ? 1 : 0;
            g.gemm.conj_a = cplx && A.conj ? 1 : 0;
            g.gemm.conj_b = cplx && B.conj ? 1 : 0;
        } else {
            // planes: 2 (bf16x3), 3 (bf16x6), or 6 exact slices with row exponents (FP64-grade)
            const int np = plan.precision == 3 ? 3 : plan.precision == 4 ? 6 : 2;
            // complex: one real GEMM of doubled K carries C = A B (4M); the
            // smaller operand is embedded (rows and K doubled), the other
            // stacked (K doubled), and the output gains a re/im digit on the
            // embedded side
            const bool emb_a = cplx && view_elems(A) <= view_elems(B);
            const int64_t Mr = cplx && emb_a ? 2 * Mx : Mx, Nr = cplx && !emb_a ? 2 * Nx : Nx;
            const int64_t Kr = cplx ? 2 * Kx : Kx;
            if (cplx) {
                cm = dbl(cm);
                cn = dbl(cn);
                if (!add_component(emb_a ? cm : cn)) return false;
            }
            TcGemmDesc &t = g.tc;
            t.M = Mr;
            t.N = Nr;
            t.bn = (Nr <= 64 || np == 6) ? 64 : (Nr <= 128 || np == 3) ? 128 : 256;
            // column tiles of the widest tile an autotuner may pick (the kernels
            // run ceil(N / bn) column tiles; the planes themselves hold N rows)
            const int bn_max = np == 6 ? 64 : np == 3 ? (Nr <= 64 ? 64 : 128) : (Nr <= 64 ? 64 : Nr <= 128 ? 128 : 256);
            t.Mp = align_up(Mr, 128);
            t.Np = align_up(Nr, bn_max);
            t.Kp = align_up(Kr, 64);
            // split K when the output tiles cannot fill the 148 SMs
            const int64_t tiles = (t.Mp / 128) * ((Nr + t.bn - 1) / t.bn), kblocks = t.Kp / 64;
            t.splitk = 1;
            if (tiles < 148 && kblocks >= 8) {
                int64_t sk = std::min<int64_t>((148 + tiles - 1) / tiles, kblocks / 4);
                if (sk > 1) t.splitk = (int)sk;
            }
            // autotuning candidates: tile width x split-K factor
            int64_t skmax = t.splitk;
            for (int bn : {64, 128, 256}) {
                if (bn > bn_max) continue;
                for (int sk : {1, 2, 4, 8, 16})
                    if (sk == 1 || (sk <= kblocks / 4 && sk * Mr * Nr * 8 <= (int64_t)512 << 20)) {
                        g.cands.push_back({bn, sk, 0});
                        skmax = std::max<int64_t>(skmax, sk);
                    }
                // an accumulating GEMM without split K may also add its tile with
                // fire-and-forget reductions (red.global.add.f64) instead of a
                // read-modify-write: no load latency in the epilogue
                if (gbeta == 1.0) g.cands.push_back({bn, 1, 1});
            }
            // the planned configuration is always one of them
            const std::array<int, 3> planned{t.bn, t.splitk, 0};
            if (std::find(g.cands.begin(), g.cands.end(), planned) == g.cands.end()) g.cands.push_back(planned);
            if (g.cands.size() < 2) g.cands.clear();
            if (skmax > 1) g.partials = scratch(skmax * Mr * Nr * 8);
            t.nplanes_a = t.nplanes_b = np;
            if (np == 2) {
                const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
                t.nprod = 3;
                for (int k = 0; k < 3; k++) { t.prod_a[k] = pa[k]; t.prod_b[k] = pb[k]; }
            } else if (np == 6) {
                t.nprod = 21;   // slice pairs (s, t) with s + t <= 5, enumerated by the kernel
            } else {
                const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
                t.nprod = 6;
                for (int k = 0; k < 6; k++) { t.prod_a[k] = pa[k]; t.prod_b[k] = pb[k]; }
            }
            t.cm = cm;
            t.cn = cn;
            t.alpha = galpha;
            t.beta = gbeta;
            SplitDesc &sa = g.split_a;
            // planes hold the real rows only: the tile padding is read as zeros by TMA
            sa.R = Mr; sa.K = Kr; sa.Rp = Mr; sa.Kp = t.Kp; sa.nplanes = np;
            sa.gr = make_grp(fa_order, A, A);
            sa.gk = make_grp(k_order, A, A);
            SplitDesc &sb = g.split_b;
            sb.R = Nr; sb.K = Kr; sb.Rp = Nr; sb.Kp = t.Kp; sb.nplanes = np;
            sb.gr = make_grp(fb_order, B, B);
            sb.gk = make_grp(k_order, B, B);
            if (cplx) {
                sa.gr = dbl(sa.gr); sa.gk = dbl(sa.gk);
                sb.gr = dbl(sb.gr); sb.gk = dbl(sb.gk);
                sa.cplx = emb_a ? 2 : 1;
                sb.cplx = emb_a ? 1 : 2;
                sa.conj = A.conj ? 1 : 0;
                sb.conj = B.conj ? 1 : 0;
            }
            g.a_static = plan.tensors[A.tensor].kind == TKind::INTEGRAL || plan.tensors[A.tensor].static_data;
            g.b_static = plan.tensors[B.tensor].kind == TKind::INTEGRAL || plan.tensors[B.tensor].static_data;
            const int64_t bytes_a = planes_bytes(Mr, t.Kp, np), bytes_b = planes_bytes(Nr, t.Kp, np);
            // static planes live in the cache; other planes in the split region, shared by
            // every later step that splits the same version of the same view
            if (g.a_static) { g.planes_a_off = cache_need; cache_need += align_up(bytes_a); }
            else { g.planes_a_off = split_slot(A.tensor, sa, g.skip_a); }
            if (g.b_static) { g.planes_b_off = cache_need; cache_need += align_up(bytes_b); }
            else { g.planes_b_off = split_slot(B.tensor, sb, g.skip_b); }
            plan.flops_mixed += flops;
        }
        plan.flops += flops;
        plan.steps.push_back(g);
        if (!direct) {
            Step e = accum_step(out, outref, Cv, cref, perms, 1.0, beta);   // alpha went into the GEMM
            if (!err.empty()) return false;
            e.stmt = si;
            e.note = "antisymmetrise -> " + T.name;
            plan.steps.push_back(e);
        }
        return true;
    }
};

}  // namespace

static bool same_ref(const BufRef &x, const BufRef &y) {
    return x.where == y.where && x.slot == y.slot && x.off == y.off;
}

// "T = X" (a plain one-term copy) directly followed by "T += alpha P(..) A * B"
// (an outer product accumulated onto T): one pass T = X + alpha sum ..., so T
// is written once and X read once instead of T being written, read and
// written again.
static void fuse_copies(Plan &plan) {
    std::vector<Step> out;
    for (size_t k = 0; k < plan.steps.size(); k++) {
        const Step &c = plan.steps[k];
        if (k + 1 < plan.steps.size()) {
            const Step &n = plan.steps[k + 1];
            const AccumDesc &a = c.acc, &b = n.acc;
            bool ok = c.kind == StepKind::ACCUM && n.kind == StepKind::ACCUM && !c.static_src && !n.static_src &&
                      !a.two_src && a.nperm == 1 && a.alpha == 1.0 && a.beta == 0.0 && a.sign[0] == 1.0 &&
                      !a.conj_a && b.two_src && b.beta == 1.0 && !b.has_add && a.cplx == b.cplx && a.nd == b.nd &&
                      same_ref(c.out, n.out) && !same_ref(n.a, n.out) && !same_ref(n.b, n.out) &&
                      !same_ref(c.a, n.out);
            for (int d = 0; ok && d < a.nd; d++) ok = a.ext[d] == b.ext[d] && a.ostr[d] == b.ostr[d];
            if (ok) {
                Step f = n;
                f.acc.has_add = 1;
                for (int d = 0; d < a.nd; d++) f.acc.astr[d] = a.sstr[0][d];
                f.c = c.a;
                f.note = c.note + " + " + n.note;
                out.push_back(f);
                k++;
                continue;
            }
        }
        out.push_back(c);
    }
    plan.steps.swap(out);
}

// K-concatenation groups.  A member is a binary contraction without permutation
// operators and without declared pairs that accumulates (+= / -=) into an
// intermediate defined earlier.  Its key is the output name and the set of
// output positions carried by the operand holding the output's innermost
// letter.  A group closes when a statement reads the output, assigns it again,
// or writes a tensor one of its members reads (so moving every member to the
// group's last position changes no operand); groups of one are dropped.
static void find_kcat_groups(const std::vector<Stmt> &stmts, const std::vector<std::vector<std::string>> &toks,
                             std::vector<std::vector<int>> &groups) {
    auto reserved = [](const std::string &n) {
        return n.empty() || n[0] == '%' || n == "V" || n == "v" || n[0] == 'T' || n[0] == 't' || n[0] == 'R' ||
               n[0] == 'r';
    };
    struct Open {
        std::string out;
        uint32_t key;
        std::vector<int> members;
        std::set<std::string> reads;
    };
    std::vector<Open> open;
    std::set<std::string> defined;
    auto close_if = [&](auto pred) {
        for (size_t g = 0; g < open.size();) {
            if (pred(open[g])) {
                if (open[g].members.size() >= 2) groups.push_back(open[g].members);
                open.erase(open.begin() + g);
            } else {
                g++;
            }
        }
    };
    for (size_t k = 0; k < stmts.size(); k++) {
        const Stmt &s = stmts[k];
        const std::string &on = s.out.name;
        // a statement reading a grouped output, or assigning it, closes its groups
        for (const Ref &r : s.rhs) close_if([&](const Open &o) { return o.out == r.name; });
        if (s.op == 0) close_if([&](const Open &o) { return o.out == on; });
        // writing a tensor a member reads closes that group
        close_if([&](const Open &o) { return o.reads.count(on) > 0; });
        bool member = s.op != 0 && s.rhs.size() == 2 && s.perms.empty() && !reserved(on) && defined.count(on) &&
                      s.rhs[0].pairs.empty() && s.rhs[1].pairs.empty() && s.rhs[0].name != on &&
                      s.rhs[1].name != on && s.out.letters.size() <= 32;
        uint32_t key = 0;
        if (member) {
            const int inner = s.out.letters.back();
            const bool a0 = std::find(s.rhs[0].letters.begin(), s.rhs[0].letters.end(), inner) != s.rhs[0].letters.end();
            const Ref &A = s.rhs[a0 ? 0 : 1], &B = s.rhs[a0 ? 1 : 0];
            bool contracted = false;
            for (int l : A.letters)
                if (std::find(B.letters.begin(), B.letters.end(), l) != B.letters.end()) contracted = true;
            member = contracted;
            for (size_t p = 0; p < s.out.letters.size(); p++)
                if (std::find(A.letters.begin(), A.letters.end(), s.out.letters[p]) != A.letters.end())
                    key |= 1u << p;
        }
        if (member) {
            Open *g = nullptr;
            for (auto &o : open)
                if (o.out == on && o.key == key) g = &o;
            if (!g) {
                open.push_back(Open{on, key, {}, {}});
                g = &open.back();
            }
            g->members.push_back((int)k);
            for (const Ref &r : s.rhs) g->reads.insert(r.name);
        }
        if (s.op == 0) defined.insert(on);
        (void)toks;
    }
    close_if([](const Open &) { return true; });
}

bool build_plan(const std::string &text, int o, int v, int dtype, int precision, Plan &plan, std::string &err,
                int flags) {
    plan = Plan();
    plan.o = o;
    plan.v = v;
    plan.packed_vvvv = (flags & 1) != 0;
    plan.dtype = dtype;
    plan.precision = precision >= 100 ? precision - 100 : precision;
    Planner P(plan);
    P.mixed_all = precision >= 100;
    P.uniform = (flags & 4) != 0;
    std::istringstream in(text);
    std::string line;
    int lineno = 0;
    int64_t max_scratch = 0;
    std::vector<Stmt> stmts;
    std::vector<std::vector<std::string>> toks;
    std::vector<std::vector<char>> spcs;
    while (std::getline(in, line)) {
        lineno++;
        size_t h = line.find('#');
        if (h != std::string::npos) line = line.substr(0, h);
        bool blank = true;
        for (char c : line)
            if (!std::isspace((unsigned char)c)) blank = false;
        if (blank) continue;
        Stmt st;
        st.line = lineno;
        std::vector<std::string> tokens;
        std::vector<char> spaces;
        std::string e;
        if (!parse_stmt(line, st, tokens, spaces, e)) {
            err = "line " + std::to_string(lineno) + ": " + e;
            return false;
        }
        plan.stmt_text.push_back(line);
        stmts.push_back(st);
        toks.push_back(tokens);
        spcs.push_back(spaces);
    }
    if (plan.stmt_text.empty()) { err = "empty contraction list"; return false; }
    // K-concatenation groups (split-route precisions, real): statements that
    // accumulate into the same intermediate with the output's letters split
    // between their operands at the same positions
    std::vector<int> group_of(stmts.size(), -1);
    std::vector<std::vector<int>> groups;
    if ((plan.precision == 2 || plan.precision == 3) && dtype == 0 && !(flags & 2)) find_kcat_groups(stmts, toks, groups);
    for (size_t g = 0; g < groups.size(); g++)
        for (int si : groups[g]) group_of[si] = (int)g;
    for (size_t k = 0; k < stmts.size(); k++) {
        const int si = (int)k;
        bool ok = true;
        if (group_of[si] >= 0) {
            if (si != groups[group_of[si]].back()) continue;   // planned with the group's last member
            // every member may run at the group's last position (the grouping
            // rule): members left out of the merge are planned there one by
            // one, in list order, and the rest merged again until it holds
            std::vector<int> gm = groups[group_of[si]];
            while (ok) {
                std::vector<const Stmt *> ms;
                std::vector<const std::vector<char> *> ls;
                for (int m : gm) { ms.push_back(&stmts[m]); ls.push_back(&spcs[m]); }
                ok = P.plan_kcat(ms, ls, gm);
                if (!ok) break;
                if (!P.kcat_declined) {
                    P.version[P.last_out] += (int)gm.size();
                    break;
                }
                P.kcat_declined = false;
                std::vector<int> rest;
                for (size_t q = 0; ok && q < gm.size(); q++) {
                    if (P.kcat_keep[q]) { rest.push_back(gm[q]); continue; }
                    ok = P.plan_stmt(stmts[gm[q]], spcs[gm[q]], gm[q]);
                    if (ok) P.version[P.last_out]++;
                    else k = gm[q];
                }
                if (!ok) break;
                if (rest.size() < 2) {
                    for (size_t q = 0; ok && q < rest.size(); q++) {
                        ok = P.plan_stmt(stmts[rest[q]], spcs[rest[q]], rest[q]);
                        if (ok) P.version[P.last_out]++;
                        else k = rest[q];
                    }
                    break;
                }
                gm = rest;
            }
        } else {
            ok = P.plan_stmt(stmts[k], spcs[k], si);
            if (ok) P.version[P.last_out]++;   // the statement's output has a new version
        }
        if (!ok) {
            err = "line " + std::to_string(stmts[k].line) + ": " + P.err;
            return false;
        }
        max_scratch = std::max(max_scratch, P.scratch_need);
    }
    fuse_copies(plan);
    // workspace: [status word][intermediates][scratch arena][static plane cache]
    plan.flags_off = 0;
    int64_t off = P.interm_need;
    plan.interm_bytes = off;
    plan.scratch_off = off;
    plan.scratch_bytes = max_scratch;
    off += max_scratch;
    plan.splits_off = off;
    plan.splits_bytes = P.splits_need;
    off += P.splits_need;
    plan.cache_off = off;
    plan.cache_bytes = P.cache_need;
    off += P.cache_need;
    plan.ws_bytes = off;
    auto place = [&](BufRef *r) {
        if (r->where == BufRef::INTEG && r->slot >= 0 && r->slot < 7) plan.integ_used[r->slot] = true;
        if (r->where == BufRef::WS && r->slot == 1) { r->off += plan.scratch_off; r->slot = 0; }
        if (r->where == BufRef::WS && r->slot == 2) { r->off += plan.cache_off; r->slot = 0; }
    };
    for (auto &st : plan.steps) {
        for (BufRef *r : {&st.out, &st.a, &st.b, &st.c, &st.partials}) place(r);
        for (KMember &m : st.kcat) { place(&m.a); place(&m.b); }
        if (st.mixed && !st.kcat.empty()) {
            st.planes_a_off += plan.scratch_off;
            st.planes_b_off += plan.scratch_off;
        } else if (st.mixed) {
            st.planes_a_off += st.a_static ? plan.cache_off : plan.splits_off;
            st.planes_b_off += st.b_static ? plan.cache_off : plan.splits_off;
        }
    }
    return true;
}

// [[bn, splitk, red], ...] of a step's autotuning candidates
static std::string cands_json(const std::vector<std::array<int, 3>> &c) {
    std::string out = "[";
    for (size_t k = 0; k < c.size(); k++)
        out += (k ? ",[" : "[") + std::to_string(c[k][0]) + "," + std::to_string(c[k][1]) + "," +
               std::to_string(c[k][2]) + "]";
    return out + "]";
}

static void grp_json(std::ostringstream &os, const Grp &g) {
    os << "{\"ext\":[";
    for (int d = 0; d < g.nd; d++) os << (d ? "," : "") << g.ext[d];
    os << "],\"str\":[";
    for (int d = 0; d < g.nd; d++) os << (d ? "," : "") << g.str[d];
    os << "]}";
}

std::string describe_plan(const Plan &plan) {
    std::ostringstream os;
    os.precision(17);
    os << "{\"o\":" << plan.o << ",\"v\":" << plan.v << ",\"dtype\":" << plan.dtype << ",\"precision\":" << plan.precision
       << ",\"workspace_bytes\":" << plan.ws_bytes << ",\"interm_bytes\":" << plan.interm_bytes
       << ",\"scratch_bytes\":" << plan.scratch_bytes << ",\"splits_bytes\":" << plan.splits_bytes
       << ",\"cache_bytes\":" << plan.cache_bytes << ",\"flops\":" << plan.flops
       << ",\"flops_mixed\":" << plan.flops_mixed << ",\"tuned\":" << (plan.tuned ? 1 : 0)
       << ",\"integrals_used\":[";
    {
        static const char *nm7[7] = {"oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv", "vvvv_packed"};
        bool first = true;
        for (int b = 0; b < 7; b++)
            if (plan.integ_used[b]) { os << (first ? "" : ",") << "\"" << nm7[b] << "\""; first = false; }
    }
    os << "],\"tensors\":[";
    for (size_t k = 0; k < plan.tensors.size(); k++) {
        const Tensor &t = plan.tensors[k];
        os << (k ? "," : "") << "{\"name\":\"" << t.name << "\",\"spaces\":\""
           << std::string(t.spaces.begin(), t.spaces.end()) << "\",\"elems\":" << t.elems << "}";
    }
    os << "],\"steps\":[";
    for (size_t k = 0; k < plan.steps.size(); k++) {
        const Step &s = plan.steps[k];
        os << (k ? "," : "") << "{\"stmt\":" << s.stmt << ",\"kind\":\""
           << (s.kind == StepKind::GEMM ? (s.mixed ? "gemm_bf16split" : s.nk ? (s.gemm.f32 ? "gemm_nk_f32" : "gemm_nk")
                                                   : s.rows ? (s.gemm.f32 ? "gemm_rows_f32" : "gemm_rows")
                                                   : s.gemm.f32 ? "gemm_f32" : "gemm_f64")
                                        : s.kind == StepKind::ACCUM ? "accum" : s.kind == StepKind::PACK ? "pack"
                                        : s.kind == StepKind::UNPACK ? "unpack" : "zero")
           << "\",\"note\":\"" << s.note << "\"";
        if (!s.kstmts.empty()) {
            os << ",\"stmts\":[";
            for (size_t q = 0; q < s.kstmts.size(); q++) os << (q ? "," : "") << s.kstmts[q];
            os << "]";
        }
        if (s.kind == StepKind::GEMM && !s.mixed) {
            os << ",\"M\":" << s.gemm.M << ",\"N\":" << s.gemm.N << ",\"K\":" << s.gemm.K << ",\"flops\":" << s.flops
               << ",\"splitk\":" << s.gemm.splitk << ",\"red\":" << (s.rows ? s.rg.red : s.gemm.red)
               << ",\"candidates\":" << s.cands.size()
               << ",\"configs\":" << cands_json(s.cands)
               << ",\"sAm\":" << s.gemm.sAm << ",\"sAk\":" << s.gemm.sAk << ",\"sBk\":" << s.gemm.sBk
               << ",\"sBn\":" << s.gemm.sBn << ",\"alpha\":" << (s.rows ? s.rg.alpha : s.gemm.alpha)
               << ",\"beta\":" << (s.rows ? s.rg.beta : s.gemm.beta)
               << ",\"conj_a\":" << s.gemm.conj_a << ",\"conj_b\":" << s.gemm.conj_b << ",\"cm\":";
            grp_json(os, s.gemm.cm);
            os << ",\"cn\":";
            grp_json(os, s.gemm.cn);
        } else if (s.kind == StepKind::GEMM) {
            int64_t K = s.split_a.K;
            if (!s.kcat.empty()) {
                K = 0;
                for (const KMember &m : s.kcat) K += m.split_a.K;
            }
            os << ",\"M\":" << s.tc.M << ",\"N\":" << s.tc.N << ",\"K\":" << K << ",\"flops\":" << s.flops
               << ",\"products\":" << s.tc.nprod << ",\"a_static\":" << (s.a_static ? 1 : 0)
               << ",\"b_static\":" << (s.b_static ? 1 : 0) << ",\"alpha\":" << s.tc.alpha << ",\"beta\":" << s.tc.beta
               << ",\"Mp\":" << s.tc.Mp << ",\"Np\":" << s.tc.Np << ",\"Kp\":" << s.tc.Kp << ",\"bn\":" << s.tc.bn
               << ",\"splitk\":" << s.tc.splitk << ",\"red\":" << s.tc.red << ",\"candidates\":" << s.cands.size()
               << ",\"configs\":" << cands_json(s.cands)
               << ",\"planes_a_off\":" << s.planes_a_off << ",\"planes_b_off\":" << s.planes_b_off
               << ",\"reuse_a\":" << (s.skip_a ? 1 : 0) << ",\"reuse_b\":" << (s.skip_b ? 1 : 0)
               << ",\"cplx_a\":" << s.split_a.cplx << ",\"cplx_b\":" << s.split_b.cplx
               << ",\"conj_a\":" << s.split_a.conj << ",\"conj_b\":" << s.split_b.conj;
        } else if (s.kind == StepKind::ACCUM) {
            os << ",\"elems\":" << s.acc.total << ",\"terms\":" << s.acc.nperm << ",\"alpha\":" << s.acc.alpha
               << ",\"beta\":" << s.acc.beta << ",\"conj_a\":" << s.acc.conj_a << ",\"conj_b\":" << s.acc.conj_b;
        } else if (s.kind == StepKind::PACK) {
            os << ",\"elems\":" << s.pk.P1 * s.pk.P2;
        } else if (s.kind == StepKind::UNPACK) {
            os << ",\"elems\":" << s.up.ext[0] * s.up.ext[1] * s.up.ext[2] * s.up.ext[3];
        } else {
            os << ",\"elems\":" << s.zero_elems;
        }
        os << "}";
    }
    os << "],\"statements\":[";
    for (size_t k = 0; k < plan.stmt_text.size(); k++) {
        std::string esc;
        for (char c : plan.stmt_text[k]) {
            if (c == '"' || c == '\\') esc += '\\';
            esc += c;
        }
        os << (k ? "," : "") << "\"" << esc << "\"";
    }
    os << "]}";
    return os.str();
}

}  // namespace ccb
