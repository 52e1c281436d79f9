// Autotune cache: launch-geometry choices measured on this GPU, stored in a
// small JSON file so that later contexts (and later processes) reuse them.
//
//   {
//     "aln_autotune": 1,
//     "entries": {
//       "<key>": {"<field>": <number>, ...},
//       ...
//     }
//   }
//
// A key names the solver path and the shape it was measured on (for example
// "single fp32 n=5000 sms=152"); the fields are the chosen parameters and the
// measurement that chose them.  The reader accepts exactly this structure
// (strings without escapes other than \" and \\, numbers); anything else makes
// the file count as empty, and the next write replaces it.  Writes go to a
// temporary file that is renamed over the cache, so a reader never sees half a
// file.
//
// What is tuned, per shape (the probes are described with each tuner below):
//   single problem     blocks and row groups of the persistent Alg. 2 kernel
//   grouped problems   the thread-block cluster size of the large problems
//   many right-hand    iterations per captured chunk and the hand-off of the
//   sides              last running columns to one block each
// Every choice only moves work between launches and blocks: each is a valid
// geometry of the same iteration, so results stay those of Alg. 2.
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace aln {
namespace {

using Fields = std::map<std::string, double>;
using Table = std::map<std::string, Fields>;

std::mutex g_tune_mutex;  // one writer at a time within the process

struct Lexer {
    const std::string& s;
    size_t i = 0;
    explicit Lexer(const std::string& t) : s(t) {}
    void ws() {
        while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    bool str(std::string* out) {
        ws();
        if (i >= s.size() || s[i] != '"') return false;
        ++i;
        out->clear();
        while (i < s.size() && s[i] != '"') {
            if (s[i] == '\\') {
                if (i + 1 >= s.size()) return false;
                const char e = s[i + 1];
                if (e != '"' && e != '\\') return false;
                out->push_back(e);
                i += 2;
            } else {
                out->push_back(s[i++]);
            }
        }
        if (i >= s.size()) return false;
        ++i;
        return true;
    }
    bool num(double* out) {
        ws();
        const char* b = s.c_str() + i;
        char* e = nullptr;
        const double v = std::strtod(b, &e);
        if (e == b) return false;
        i += (size_t)(e - b);
        *out = v;
        return true;
    }
};

bool parse(const std::string& text, Table* t) {
    Lexer L(text);
    if (!L.eat('{')) return false;
    bool have_entries = false;
    for (;;) {
        std::string k;
        if (!L.str(&k) || !L.eat(':')) return false;
        if (k == "entries") {
            if (!L.eat('{')) return false;
            if (!L.eat('}')) {
                for (;;) {
                    std::string key;
                    if (!L.str(&key) || !L.eat(':') || !L.eat('{')) return false;
                    Fields f;
                    if (!L.eat('}')) {
                        for (;;) {
                            std::string name;
                            double v = 0.0;
                            if (!L.str(&name) || !L.eat(':') || !L.num(&v)) return false;
                            f[name] = v;
                            if (L.eat('}')) break;
                            if (!L.eat(',')) return false;
                        }
                    }
                    (*t)[key] = f;
                    if (L.eat('}')) break;
                    if (!L.eat(',')) return false;
                }
            }
            have_entries = true;
        } else {
            double v = 0.0;
            if (!L.num(&v)) return false;
        }
        if (L.eat('}')) break;
        if (!L.eat(',')) return false;
    }
    return have_entries;
}

std::string quote(const std::string& s) {
    std::string o = "\"";
    for (char ch : s) {
        if (ch == '"' || ch == '\\') o.push_back('\\');
        o.push_back(ch);
    }
    return o + "\"";
}

std::string render(const Table& t) {
    std::ostringstream o;
    o.precision(17);
    o << "{\n  \"aln_autotune\": 1,\n  \"entries\": {";
    bool first = true;
    for (const auto& e : t) {
        o << (first ? "\n" : ",\n") << "    " << quote(e.first) << ": {";
        bool f2 = true;
        for (const auto& f : e.second) {
            o << (f2 ? "" : ", ") << quote(f.first) << ": " << f.second;
            f2 = false;
        }
        o << "}";
        first = false;
    }
    o << "\n  }\n}\n";
    return o.str();
}

Table load(const std::string& path) {
    Table t;
    std::ifstream in(path, std::ios::binary);
    if (!in) return t;
    std::stringstream ss;
    ss << in.rdbuf();
    if (!parse(ss.str(), &t)) t.clear();
    return t;
}

}  // namespace


namespace {

#define T_TRY(call)                                       \
    do {                                                  \
        if ((call) != cudaSuccess) {                      \
            cudaGetLastError();                           \
            return ALN_ERR_CUDA;                          \
        }                                                 \
    } while (0)
#define T_CHECK(call)                 \
    do {                              \
        aln_status s_ = (call);       \
        if (s_ != ALN_OK) return s_;  \
    } while (0)

bool lookup(const aln_ctx* c, const std::string& key, Fields* out) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const Table t = load(c->tune_path);
    const auto e = t.find(key);
    if (e == t.end()) return false;
    *out = e->second;
    return true;
}

bool get(const Fields& f, const char* name, double* v) {
    const auto it = f.find(name);
    if (it == f.end() || !(it->second == it->second)) return false;
    *v = it->second;
    return true;
}

// Adds (or replaces) one entry; the file is re-read under the lock so that
// entries written by other contexts since are kept.
bool record(const aln_ctx* c, const std::string& key, const Fields& f) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    Table t = load(c->tune_path);
    t[key] = f;
    const std::string tmp = c->tune_path + ".tmp";
    {
        std::ofstream out(tmp, std::ios::binary | std::ios::trunc);
        if (!out) return false;
        out << render(t);
        if (!out) return false;
    }
    return std::rename(tmp.c_str(), c->tune_path.c_str()) == 0;
}

// Two events on the context's stream around a region.
struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
            cudaGetLastError();
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    bool ok() const { return a && b; }
};

std::string prec_name(const aln_ctx* c) {
    return c->opt.precision == ALN_PREC_FP64 ? "fp64" : "split_bf16";
}

// ---------------------------------------------------------------------------
// Single problem: blocks G and row groups R of the persistent Alg. 2 kernel
// (work items = column tiles × R, dealt round-robin to G co-resident blocks).
// Probe: Alg. 2 from y = 0 on the first right-hand side with eps = 0, so every
// candidate runs the same kProbeIters iterations; the score is the time per
// iteration, best of two runs.
constexpr int kProbeIters = 64;

aln_status set_geometry(aln_ctx* c, int G, int R) {
    c->opt.persist_blocks = G;
    c->tune_pR = R;
    return alloc_workspace(c);
}

aln_status single_probe(aln_ctx* c, double* us_per_iter) {
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    T_TRY(f64 ? launch_iter_setup<double>(c, c->q64, nullptr, 0.0, kProbeIters)
              : launch_iter_setup<float>(c, c->q64, nullptr, 0.0, kProbeIters));
    c->launches += 3;
    const double before = c->stats.iterate_ms;
    T_CHECK(run_until_done(c));
    const int it = c->st_host->iter;
    // an early stop (empty passive set) leaves nothing to compare
    *us_per_iter = it >= kProbeIters / 2 ? 1e3 * (c->stats.iterate_ms - before) / it : -1.0;
    return ALN_OK;
}

aln_status tune_single(aln_ctx* c) {
    if (c->opt.algorithm != ALN_ALG_ANTILOP || c->p_small || c->k < 1) return ALN_OK;
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    char buf[192];
    snprintf(buf, sizeof buf, "single %s n=%lld sms=%d kernel=%s", prec_name(c).c_str(),
             (long long)c->n, c->num_sms, c->p_repl ? "replicated" : "tiled");
    const std::string key = buf;
    if (c->tuned_key == key) return ALN_OK;
    const int S = c->num_sms, CT = c->p_CT;
    const int rmax = (int)std::min<int64_t>(64, ceil_div(c->n, 32));
    int repl = c->p_repl;
    const int maxG = f64 ? persist_max_blocks<double>(S, c->ldq, &repl)
                         : persist_max_blocks<float>(S, c->ldq, &repl);
    if (maxG <= 0) return ALN_ERR_CUDA;
    Fields f;
    double G = 0.0, R = 0.0;
    if (lookup(c, key, &f) && get(f, "persist_blocks", &G) && get(f, "row_groups", &R) &&
        G >= 1.0 && G <= maxG && R >= 1.0 && R <= rmax) {
        T_CHECK(set_geometry(c, (int)G, (int)R));
        c->tuned_key = key;
        return ALN_OK;
    }
    const int G0 = c->user_opt.persist_blocks;
    if (c->opt.autotune < 2) {  // no choice cached: the caller's geometry
        if (c->opt.persist_blocks != G0 || c->tune_pR != 0) T_CHECK(set_geometry(c, G0, 0));
        c->tuned_key = key;
        return ALN_OK;
    }
    // candidates: the default geometry first, then every R whose CT·R work
    // items are between S/2 and 3S, each with one or two items per block
    std::vector<std::pair<int, int>> cand{{G0, 0}};
    auto add = [&](int64_t g, int r) {
        g = std::min<int64_t>(g, maxG);
        if (g < 1) return;
        for (const auto& p : cand)
            if (p.first == (int)g && p.second == r) return;
        cand.push_back({(int)g, r});
    };
    for (int r = 1; r <= rmax; ++r) {
        const int64_t items = (int64_t)CT * r;
        if (items < S / 2 && r < rmax) continue;
        if (items > 3LL * S) break;
        add(items, r);
        if (ceil_div(items, 2) >= S / 4) add(ceil_div(items, 2), r);
    }
    std::vector<double> score(cand.size(), -1.0);
    double us = 0.0;
    T_CHECK(set_geometry(c, G0, 0));
    T_CHECK(single_probe(c, &us));  // warm-up (first launches, caches)
    if (us < 0.0) {  // the probe stopped early: keep the default, record nothing
        c->tuned_key = key;
        return ALN_OK;
    }
    size_t best = 0;
    for (size_t i = 0; i < cand.size(); ++i) {
        T_CHECK(set_geometry(c, cand[i].first, cand[i].second));
        if (c->p_G != (cand[i].first > 0 ? cand[i].first : c->p_G) ||
            (cand[i].second > 0 && c->p_R != cand[i].second))
            continue;  // clamped by the workspace rules: not this geometry
        double t = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            T_CHECK(single_probe(c, &us));
            if (us > 0.0) t = std::min(t, us);
        }
        score[i] = t < 1e300 ? t : -1.0;
        if (score[i] > 0.0 && (score[best] < 0.0 || score[i] < score[best])) best = i;
    }
    // record the geometry actually in force for the winner
    T_CHECK(set_geometry(c, cand[best].first, cand[best].second));
    const int bestG = c->p_G, bestR = c->p_R;
    T_CHECK(set_geometry(c, bestG, bestR));
    if (score[best] > 0.0)
        record(c, key,
               {{"persist_blocks", (double)bestG}, {"row_groups", (double)bestR},
                {"us_per_iter", score[best]}, {"default_us_per_iter", score[0]},
                {"candidates", (double)cand.size()}, {"probe_iters", (double)kProbeIters}});
    c->tuned_key = key;
    return ALN_OK;
}

// ---------------------------------------------------------------------------
// Grouped problems: the thread-block cluster size of the large problems.
// Probe: the whole solve with the caller's tol and max_iter (host-driven
// rounds), once per cluster size after a warm-up; the result is overwritten
// by the solve that follows.
aln_status tune_grouped(aln_ctx* c, double tol, int max_iter, double* X, const double* X0) {
    int count = 0;
    int64_t sum_n = 0, max_n = 0;
    group_shape(c, &count, &sum_n, &max_n);
    char buf[192];
    snprintf(buf, sizeof buf, "grouped %s count=%d sum_n=%lld max_n=%lld sms=%d",
             prec_name(c).c_str(), count, (long long)sum_n, (long long)max_n, c->num_sms);
    const std::string key = buf;
    if (c->tuned_key == key) return ALN_OK;
    Fields f;
    double cs = 0.0;
    if (lookup(c, key, &f) && get(f, "group_cluster", &cs) &&
        (cs == 1.0 || cs == 2.0 || cs == 4.0 || cs == 8.0)) {
        c->opt.group_cluster = (int)cs;
        c->tuned_key = key;
        return ALN_OK;
    }
    c->opt.group_cluster = c->user_opt.group_cluster;
    if (c->opt.autotune < 2) {
        c->tuned_key = key;
        return ALN_OK;
    }
    Timer tm;
    if (!tm.ok()) return ALN_ERR_CUDA;
    const int graph = c->opt.group_graph;
    c->opt.group_graph = 0;
    auto timed = [&](int size, float* ms) -> aln_status {
        c->opt.group_cluster = size;
        T_TRY(cudaEventRecord(tm.a, c->stream));
        T_CHECK(group_solve(c, tol, max_iter, X, X0, nullptr));
        T_TRY(cudaEventRecord(tm.b, c->stream));
        T_TRY(cudaEventSynchronize(tm.b));
        T_TRY(cudaEventElapsedTime(ms, tm.a, tm.b));
        return ALN_OK;
    };
    const int sizes[4] = {1, 2, 4, 8};
    float ms[4] = {0, 0, 0, 0}, warm = 0.f, dflt = 0.f;
    aln_status st = timed(c->user_opt.group_cluster, &warm);
    if (st == ALN_OK) st = timed(c->user_opt.group_cluster, &dflt);
    int best = -1;
    for (int i = 0; i < 4 && st == ALN_OK; ++i) {
        st = timed(sizes[i], &ms[i]);
        if (st == ALN_OK && (best < 0 || ms[i] < ms[best])) best = i;
    }
    c->opt.group_graph = graph;
    if (st != ALN_OK) {
        c->opt.group_cluster = c->user_opt.group_cluster;
        return st;
    }
    c->opt.group_cluster = sizes[best];
    record(c, key,
           {{"group_cluster", (double)sizes[best]}, {"solve_ms", (double)ms[best]},
            {"default_solve_ms", (double)dflt}, {"cluster1_ms", (double)ms[0]},
            {"cluster2_ms", (double)ms[1]}, {"cluster4_ms", (double)ms[2]},
            {"cluster8_ms", (double)ms[3]}});
    c->tuned_key = key;
    return ALN_OK;
}

// ---------------------------------------------------------------------------
// Many right-hand sides: iterations per captured chunk (how often the host
// reads the running count) and the number of running columns below which the
// rest go to one block each.  Probe: whole solves, chunk first (hand-off at
// its default), then the hand-off at the best chunk.
aln_status tune_batched(aln_ctx* c, double tol, int max_iter, double* X, int64_t ldx,
                        const double* X0) {
    if (c->n <= 128) return ALN_OK;  // one warp per column: no chunks, no hand-off
    char buf[192];
    snprintf(buf, sizeof buf, "batched %s n=%lld k=%lld sms=%d", prec_name(c).c_str(),
             (long long)c->n, (long long)c->k, c->num_sms);
    const std::string key = buf;
    if (c->tuned_key == key) return ALN_OK;
    const int S = c->num_sms;
    Fields f;
    double ch = 0.0, tl = 0.0;
    if (lookup(c, key, &f) && get(f, "chunk", &ch) && get(f, "handoff", &tl) && ch >= 1.0 &&
        ch <= 64.0 && tl >= 1.0 && tl <= 64.0 * S) {
        c->tune_chunk = (int)ch;
        c->tune_tail = (int)tl;
        double bu = 0.0;  // optional: iterations per tail launch
        c->tune_budget = get(f, "tail_budget", &bu) && bu >= 1.0 && bu <= 1e6 ? (int)bu : 0;
        c->tuned_key = key;
        return ALN_OK;
    }
    c->tune_chunk = c->tune_tail = c->tune_budget = 0;
    if (c->opt.autotune < 2) {
        c->tuned_key = key;
        return ALN_OK;
    }
    Timer tm;
    if (!tm.ok()) return ALN_ERR_CUDA;
    auto timed = [&](int chunk, int tail, float* ms) -> aln_status {
        c->tune_chunk = chunk;
        c->tune_tail = tail;
        T_TRY(cudaEventRecord(tm.a, c->stream));
        T_CHECK(batch_solve(c, tol, max_iter, X, ldx, X0, nullptr));
        T_TRY(cudaEventRecord(tm.b, c->stream));
        T_TRY(cudaEventSynchronize(tm.b));
        T_TRY(cudaEventElapsedTime(ms, tm.a, tm.b));
        return ALN_OK;
    };
    float warm = 0.f, dflt = 0.f;
    aln_status st = timed(8, 2 * S, &warm);
    if (st == ALN_OK) st = timed(8, 2 * S, &dflt);
    int bc = 8, bt = 2 * S;
    float bms = dflt;
    for (int chunk : {4, 16, 32}) {
        float ms = 0.f;
        if (st == ALN_OK) st = timed(chunk, 2 * S, &ms);
        if (st == ALN_OK && ms < bms) {
            bms = ms;
            bc = chunk;
        }
    }
    for (int tail : {S, 4 * S}) {
        float ms = 0.f;
        if (st == ALN_OK) st = timed(bc, tail, &ms);
        if (st == ALN_OK && ms < bms) {
            bms = ms;
            bt = tail;
        }
    }
    if (st != ALN_OK) {
        c->tune_chunk = c->tune_tail = 0;
        return st;
    }
    c->tune_chunk = bc;
    c->tune_tail = bt;
    record(c, key,
           {{"chunk", (double)bc}, {"handoff", (double)bt}, {"solve_ms", (double)bms},
            {"default_solve_ms", (double)dflt}});
    c->tuned_key = key;
    return ALN_OK;
}

}  // namespace

aln_status autotune_solve(aln_ctx* c, double tol, int max_iter, double* X, int64_t ldx,
                          const double* X0) {
    if (c->opt.autotune == 0 || c->tune_path.empty()) return ALN_OK;
    const aln_stats saved = c->stats;
    aln_status st = c->grouped   ? tune_grouped(c, tol, max_iter, X, X0)
                    : c->batched ? tune_batched(c, tol, max_iter, X, ldx, X0)
                                 : tune_single(c);
    c->stats = saved;
    return st;
}

}  // namespace aln
