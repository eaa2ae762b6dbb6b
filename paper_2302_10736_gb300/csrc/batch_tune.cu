// batch_tune.cu - launch configuration of batches (no counterpart in the
// paper): get/set, the autotuner of the batched launches, and its cache, a
// JSON file keyed by GPU name, kernel family and size class.
//
// The configuration does not change results beyond the rounding of loss sums:
// every bus and Jacobian entry is summed over the same terminals in the same
// order whatever the windows, so the tuner only trades launch shapes.
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "pf_internal.h"

namespace pf {
namespace {

// ---------------------------------------------------------- the cache file --
// {"pfgrid_tune_cache": 1, "entries": {"<key>": {"window": 256, ...}, ...}}
using Fields = std::map<std::string, double>;
using Entries = std::map<std::string, Fields>;

const char *const kFieldNames[] = {"window", "terminals_per_thread", "ctas_per_sm", "adjoint_form", "ybus_lanes",
                                   "ybus_block"};

Fields to_fields(const pf_batch_config &c)
{
    const int32_t v[] = {c.window, c.terminals_per_thread, c.ctas_per_sm, c.adjoint_form, c.ybus_lanes, c.ybus_block};
    Fields f;
    for (int i = 0; i < 6; ++i) f[kFieldNames[i]] = v[i];
    return f;
}

bool from_fields(const Fields &f, pf_batch_config &c)
{
    int32_t *v[] = {&c.window, &c.terminals_per_thread, &c.ctas_per_sm, &c.adjoint_form, &c.ybus_lanes, &c.ybus_block};
    for (int i = 0; i < 6; ++i) {
        auto it = f.find(kFieldNames[i]);
        if (it == f.end()) return false;
        *v[i] = (int32_t)it->second;
    }
    return true;
}

// A small recursive-descent reader for the subset of JSON the cache uses:
// objects, strings without escapes, numbers; other values are skipped.
struct Reader {
    const std::string &s;
    size_t i = 0;
    bool ok = true;
    explicit Reader(const std::string &str) : s(str) {}
    void ws()
    {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
    }
    bool eat(char c)
    {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    std::string str()
    {
        ws();
        std::string out;
        if (i >= s.size() || s[i] != '"') {
            ok = false;
            return out;
        }
        ++i;
        while (i < s.size() && s[i] != '"') {
            if (s[i] == '\\') {   // escapes are not produced by the writer
                ok = false;
                return out;
            }
            out += s[i++];
        }
        if (i >= s.size()) ok = false;
        ++i;
        return out;
    }
    double num()
    {
        ws();
        const char *p = s.c_str() + i;
        char *end = nullptr;
        const double v = std::strtod(p, &end);
        if (end == p) ok = false;
        i += (size_t)(end - p);
        return v;
    }
    void skip_value()
    {
        ws();
        if (i >= s.size()) {
            ok = false;
            return;
        }
        const char c = s[i];
        if (c == '{') {
            Fields dummy;
            object_of_numbers(dummy, true);
        } else if (c == '"') {
            str();
        } else if (c == '[') {
            ++i;
            if (eat(']')) return;
            do skip_value();
            while (ok && eat(','));
            if (!eat(']')) ok = false;
        } else if (c == 't' || c == 'f' || c == 'n') {
            while (i < s.size() && isalpha((unsigned char)s[i])) ++i;
        } else {
            num();
        }
    }
    // {"name": number, ...}; with `lenient`, non-numeric members are skipped
    void object_of_numbers(Fields &f, bool lenient)
    {
        if (!eat('{')) {
            ok = false;
            return;
        }
        if (eat('}')) return;
        do {
            const std::string k = str();
            if (!ok || !eat(':')) {
                ok = false;
                return;
            }
            ws();
            if (i < s.size() && (s[i] == '-' || isdigit((unsigned char)s[i])))
                f[k] = num();
            else if (lenient)
                skip_value();
            else
                ok = false;
        } while (ok && eat(','));
        if (ok && !eat('}')) ok = false;
    }
};

// Missing file: empty cache (true).  Unreadable or malformed: false.
bool read_cache(const char *path, Entries &e)
{
    e.clear();
    FILE *f = std::fopen(path, "rb");
    if (!f) return true;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
    std::fclose(f);
    Reader r(txt);
    if (!r.eat('{')) return false;
    if (r.eat('}')) return true;
    do {
        const std::string k = r.str();
        if (!r.ok || !r.eat(':')) return false;
        if (k == "entries") {
            if (!r.eat('{')) return false;
            if (!r.eat('}')) {
                do {
                    const std::string key = r.str();
                    if (!r.ok || !r.eat(':')) return false;
                    Fields fl;
                    r.object_of_numbers(fl, true);
                    if (!r.ok) return false;
                    e[key] = fl;
                } while (r.eat(','));
                if (!r.eat('}')) return false;
            }
        } else {
            r.skip_value();
            if (!r.ok) return false;
        }
    } while (r.eat(','));
    return r.eat('}');
}

bool write_cache(const char *path, const Entries &e)
{
    const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    std::fprintf(f, "{\n  \"pfgrid_tune_cache\": 1,\n  \"entries\": {");
    bool first = true;
    for (const auto &kv : e) {
        std::fprintf(f, "%s\n    \"%s\": {", first ? "" : ",", kv.first.c_str());
        bool ff = true;
        for (const auto &fv : kv.second) {
            std::fprintf(f, "%s\"%s\": %.17g", ff ? "" : ", ", fv.first.c_str(), fv.second);
            ff = false;
        }
        std::fprintf(f, "}");
        first = false;
    }
    std::fprintf(f, "\n  }\n}\n");
    const bool ok = std::fflush(f) == 0 && std::ferror(f) == 0;
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

bool key_ok(const char *key) { return key && *key && !std::strpbrk(key, "\"\\"); }

int pow2_at_least(long long x)
{
    int p = 0;
    while ((1LL << p) < x) ++p;
    return p;
}

std::string tune_key(const Batch *b)
{
    int dev = 0;
    cudaDeviceProp prop{};
    std::string name = "unknown-gpu";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == '"' || c == '\\') c = '_';
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|batched|nb<=2^%d|S<=2^%d|%s", name.c_str(), pow2_at_least(b->g->nb),
                  pow2_at_least(b->S), b->has_outage ? "n-1" : "no-outage");
    return buf;
}

const char *cache_path() { return std::getenv("PFGRID_TUNE_CACHE"); }

pf_status check_config(const pf_batch_config &c)
{
    if (c.window != 128 && c.window != 256) return set_error(PF_EINVAL, "batch config: window = %d", c.window);
    if (c.terminals_per_thread < 1 || c.terminals_per_thread > 3)
        return set_error(PF_EINVAL, "batch config: terminals_per_thread = %d", c.terminals_per_thread);
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 8) return set_error(PF_EINVAL, "batch config: ctas_per_sm = %d", c.ctas_per_sm);
    if (c.adjoint_form != 0 && c.adjoint_form != 1)
        return set_error(PF_EINVAL, "batch config: adjoint_form = %d", c.adjoint_form);
    const int l = c.ybus_lanes;
    if (l != 1 && l != 2 && l != 4 && l != 8 && l != 16 && l != 32)
        return set_error(PF_EINVAL, "batch config: ybus_lanes = %d", l);
    if (c.ybus_block < 32 || c.ybus_block > 512 || c.ybus_block % 32)
        return set_error(PF_EINVAL, "batch config: ybus_block = %d", c.ybus_block);
    return PF_OK;
}

}  // namespace

pf_status batch_apply_config(Batch *b, const pf_batch_config &c, cudaStream_t st)
{
    if (pf_status e = check_config(c)) return e;
    if (c.window != b->tb || c.terminals_per_thread != b->tfac) {
        HostEw E;
        bool ghost = false;
        if (pf_status e = batch_plan(b->g, b->S, c.window, c.terminals_per_thread, E, ghost)) return e;
        if (pf_status e = batch_upload(b, E, ghost, st)) return e;
    }
    b->cfg = c;
    b->cfg.terminals_per_thread = b->tfac;
    return PF_OK;
}

pf_status batch_apply_cached(Batch *b, cudaStream_t st)
{
    const char *path = cache_path();
    if (!path || !*path) return PF_OK;
    Entries e;
    if (!read_cache(path, e)) return PF_OK;   // the cache is an optimisation: a bad file is ignored
    auto it = e.find(tune_key(b));
    pf_batch_config c{};
    if (it == e.end() || !from_fields(it->second, c) || check_config(c) != PF_OK) return PF_OK;
    return batch_apply_config(b, c, st);
}

}  // namespace pf

using namespace pf;

PF_API pf_status pf_tune_cache_lookup(const char *path, const char *key, pf_batch_config *cfg, int32_t *found)
{
    if (!path || !key || !cfg || !found) return set_error(PF_EINVAL, "pf_tune_cache_lookup: NULL argument");
    *found = 0;
    if (!key_ok(key)) return set_error(PF_EINVAL, "pf_tune_cache_lookup: invalid key");
    Entries e;
    if (!read_cache(path, e)) return set_error(PF_EINVAL, "pf_tune_cache_lookup: %s is not a tuning cache", path);
    auto it = e.find(key);
    if (it == e.end()) return PF_OK;
    pf_batch_config c{};
    if (!from_fields(it->second, c)) return set_error(PF_EINVAL, "pf_tune_cache_lookup: entry %s incomplete", key);
    *cfg = c;
    *found = 1;
    return PF_OK;
}

PF_API pf_status pf_tune_cache_store(const char *path, const char *key, const pf_batch_config *cfg)
{
    if (!path || !key || !cfg) return set_error(PF_EINVAL, "pf_tune_cache_store: NULL argument");
    if (!key_ok(key)) return set_error(PF_EINVAL, "pf_tune_cache_store: invalid key");
    Entries e;
    if (!read_cache(path, e)) return set_error(PF_EINVAL, "pf_tune_cache_store: %s is not a tuning cache", path);
    e[key] = to_fields(*cfg);
    if (!write_cache(path, e)) return set_error(PF_EINVAL, "pf_tune_cache_store: cannot write %s", path);
    return PF_OK;
}

PF_API pf_status batch_tune_key(const pf_batch *batch, char *buf, int32_t len)
{
    if (!batch || !buf || len <= 0) return set_error(PF_EINVAL, "batch_tune_key: NULL or empty buffer");
    const std::string k = tune_key(&batch->b);
    if ((int32_t)k.size() >= len) return set_error(PF_EINVAL, "batch_tune_key: buffer of %d bytes too small", len);
    std::memcpy(buf, k.c_str(), k.size() + 1);
    return PF_OK;
}

PF_API pf_status batch_get_config(const pf_batch *batch, pf_batch_config *cfg)
{
    if (!batch || !cfg) return set_error(PF_EINVAL, "batch_get_config: NULL argument");
    *cfg = batch->b.cfg;
    return PF_OK;
}

PF_API pf_status batch_set_config(pf_batch *batch, const pf_batch_config *cfg, pf_stream stream)
{
    if (!batch || !cfg) return set_error(PF_EINVAL, "batch_set_config: NULL argument");
    return batch_apply_config(&batch->b, *cfg, (cudaStream_t)stream);
}

namespace {

// mean ms per launch of fn over reps launches after one untimed launch
template <typename F>
pf_status time_launches(F fn, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    if (pf_status st = fn()) return st;
    PF_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r)
        if (pf_status st = fn()) return st;
    PF_CUDA(cudaEventRecord(e1, s));
    PF_CUDA(cudaEventSynchronize(e1));
    PF_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= (float)reps;
    return PF_OK;
}

}  // namespace

PF_API pf_status batch_autotune(pf_batch *batch, const double *vm, const double *va, int32_t kernels, int32_t reps,
                                pf_stream stream, pf_batch_config *best)
{
    if (!batch || !vm || !va) return set_error(PF_EINVAL, "batch_autotune: NULL argument");
    if (reps < 1) return set_error(PF_EINVAL, "batch_autotune: reps = %d", reps);
    if (kernels == 0) kernels = PF_TUNE_JAC | PF_TUNE_YBUS;
    if (kernels & ~(PF_TUNE_JAC | PF_TUNE_YBUS | PF_TUNE_ADJOINT))
        return set_error(PF_EINVAL, "batch_autotune: kernels = %d", kernels);
    Batch *b = &batch->b;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->S == 0 || b->g->nb == 0) {
        if (best) *best = b->cfg;
        return PF_OK;
    }
    const size_t n = (size_t)b->S * b->g->nb;
    const int nb = b->g->nb, nl = b->g->nl;
    double *P = nullptr, *Q = nullptr, *J = nullptr, *spec = nullptr, *grads = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pf_status st = PF_OK;
    pf_batch_config cur = b->cfg, win = b->cfg;
    float best_ms = 0.0f;
    bool have = false;
    auto cleanup = [&]() {
        cudaFree(P);
        cudaFree(Q);
        cudaFree(J);
        cudaFree(spec);
        cudaFree(grads);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t ce;
    if ((ce = cudaMalloc(&P, n * sizeof(double))) || (ce = cudaMalloc(&Q, n * sizeof(double))) ||
        (ce = cudaMalloc(&J, std::max<long long>(b->h_joff.back(), 1) * sizeof(double))) ||
        (ce = cudaEventCreate(&e0)) || (ce = cudaEventCreate(&e1)) ||
        // the adjoint's inputs (targets 0, weights 1: its cost does not depend on
        // their values) and outputs
        ((kernels & PF_TUNE_ADJOINT) &&
         ((ce = cudaMalloc(&spec, 4 * (size_t)nb * sizeof(double))) ||
          (ce = cudaMemsetAsync(spec, 0, 2 * (size_t)nb * sizeof(double), s)) ||
          (ce = cudaMalloc(&grads, (2 * n + 4 * (size_t)nl + b->S + 1) * sizeof(double)))))) {
        cleanup();
        return cuda_error(ce, "batch_autotune");
    }
    if (kernels & PF_TUNE_ADJOINT) {   // weights of 1.0 (the bytes of 1.0 are not a repeated byte)
        std::vector<double> ones(2 * (size_t)nb, 1.0);
        if ((ce = cudaMemcpyAsync(spec + 2 * (size_t)nb, ones.data(), ones.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, s)) ||
            (ce = cudaStreamSynchronize(s))) {
            cleanup();
            return cuda_error(ce, "batch_autotune");
        }
    }
    auto ew = [&]() -> pf_status {
        if (kernels & PF_TUNE_JAC) {
            TraceScope t(b->g, PF_K_JAC_EW_BATCHED, s);
            PF_CUDA(launch_ew_batched(b, true, vm, va, P, Q, J, s));
        }
        if (kernels & PF_TUNE_ADJOINT) {
            const size_t nbz = (size_t)nb;
            double *gvm = grads, *gva = grads + n, *gp = grads + 2 * n;
            TraceScope t(b->g, PF_K_ADJOINT, s);
            PF_CUDA(launch_adjoint(b, vm, va, spec, spec + nbz, spec + 2 * nbz, spec + 3 * nbz, nullptr,
                                   gp + 4 * (size_t)nl, gp + 4 * (size_t)nl + b->S, gvm, gva, gp, gp + nl,
                                   gp + 2 * (size_t)nl, gp + 3 * (size_t)nl, s));
        }
        return PF_OK;
    };
    auto yb = [&]() -> pf_status {
        TraceScope t(b->g, PF_K_JAC_YBUS_BATCHED, s);
        PF_CUDA(launch_ybus_batched(b, true, vm, va, P, Q, J, s));
        return PF_OK;
    };
    // element-wise: window size x terminal cap x CTAs per SM (x the adjoint's
    // form when the adjoint is tuned), by the total time of the selected kernels
    for (int window : {128, 256}) {
        if (!(kernels & (PF_TUNE_JAC | PF_TUNE_ADJOINT))) break;
        for (int tpt = 1; tpt <= 3; ++tpt) {
            pf_batch_config c = cur;
            c.window = window;
            c.terminals_per_thread = tpt;
            c.ctas_per_sm = 0;
            st = batch_apply_config(b, c, s);
            if (st == PF_EUNSUPPORTED) {   // this window shape does not fit in shared memory
                st = PF_OK;
                continue;
            }
            if (st) break;
            for (int cps : {0, 1, 2, 3}) {
                for (int form = 0; form < ((kernels & PF_TUNE_ADJOINT) ? 2 : 1); ++form) {
                    b->cfg.ctas_per_sm = cps;
                    b->cfg.adjoint_form = (kernels & PF_TUNE_ADJOINT) ? form : cur.adjoint_form;
                    float ms = 0.0f;
                    if ((st = time_launches(ew, reps, s, e0, e1, &ms))) break;
                    if (!have || ms < best_ms) {
                        best_ms = ms;
                        win = b->cfg;
                        have = true;
                    }
                }
                if (st) break;
            }
            if (st) break;
        }
        if (st) break;
    }
    // the batched Ybus method: lanes per row x CTA size (independent of the windows)
    if (st == PF_OK && (st = batch_apply_config(b, win, s)) == PF_OK && (kernels & PF_TUNE_YBUS)) {
        float yb_best = 0.0f;
        bool yhave = false;
        pf_batch_config ywin = win;
        for (int lanes : {1, 2, 4, 8, 16, 32}) {
            for (int blk : {128, 256, 512}) {
                b->cfg.ybus_lanes = lanes;
                b->cfg.ybus_block = blk;
                float ms = 0.0f;
                if ((st = time_launches(yb, reps, s, e0, e1, &ms))) break;
                if (!yhave || ms < yb_best) {
                    yb_best = ms;
                    ywin = b->cfg;
                    yhave = true;
                }
            }
            if (st) break;
        }
        win.ybus_lanes = ywin.ybus_lanes;
        win.ybus_block = ywin.ybus_block;
    }
    cleanup();
    if (st) {
        batch_apply_config(b, cur, s);   // leave the batch as it was
        return st;
    }
    if ((st = batch_apply_config(b, win, s))) return st;
    if (best) *best = b->cfg;
    const char *path = cache_path();
    if (path && *path) {
        const std::string key = tune_key(b);
        if ((st = pf_tune_cache_store(path, key.c_str(), &b->cfg))) return st;
    }
    return PF_OK;
}
