// Tuning registry (see tune.hpp).
#include "tune.hpp"

#include <dlfcn.h>

#include <atomic>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.hpp"

namespace hxc {
namespace tune {
namespace {

struct Knob {
    const char *key;
    int64_t value, lo, hi;
};

// key, default, min, max
Knob g_knobs[] = {
    {"heat2d.emul", 0, 0, 4},         // integer-pipe share of the 2D additions
    {"heat2d.rows", 16, 1, 4096},     // rows per warp of the 2D kernel
    {"heat2d.occupancy", 4, 4, 6},    // compiled minimum of CTAs per SM
    {"heat3d.zchunks", 0, 0, 64},     // z chunks per launch of form 2 (0: fill whole waves)
    {"heat3d.variant", 6, 2, 7},      // 2 three-plane, 3 two-plane, 4 + ring, 6 + packed narrow tiles, 7 + TMA
    {"heat3d.variant1", 5, 2, 7},     // the same choice for one-step launches, 5 = streaming one-step kernel
    {"heat1d.tb_ctas", 0, 0, 1 << 16},  // CTAs per partition of the 1D blocked kernel (0: SMs/parts)
    {"heat1d.steps_per_launch", 0, 0, 1024},  // fused 1D steps per launch when the caller passes 0 (0: all)
    {"heat3d.steps_per_launch", 4, 1, 4},     // fused 3D steps per launch when the caller passes 0
    {"mandel.pair", 1, 0, 1},         // Mandelbrot: 1 = two pixels per thread on paired FP32
    {"batch.ctas_per_sm", 4, 1, 16},  // CTAs per SM of the persistent batch kernel
    {"batch.block", 256, 256, 1024},  // threads per CTA of the persistent batch kernel
    {"batch.smem_side", 0, 0, 119},   // largest side kept in shared memory for a whole run (0: none)
};
std::mutex g_m;

Knob *find(const char *key) {
    if (!key) return nullptr;
    for (auto &k : g_knobs)
        if (strcmp(k.key, key) == 0) return &k;
    return nullptr;
}

// Minimal reader for {"a": {"k": 1, ...}, "b": ...} or {"k": 1, ...}.
struct Reader {
    const char *p, *e;
    void ws() {
        while (p < e && isspace((unsigned char)*p)) p++;
    }
    bool ch(char c) {
        ws();
        if (p < e && *p == c) {
            p++;
            return true;
        }
        return false;
    }
    bool str(std::string *out) {
        ws();
        if (p >= e || *p != '"') return false;
        p++;
        out->clear();
        while (p < e && *p != '"') out->push_back(*p++);
        if (p >= e) return false;
        p++;
        return true;
    }
    bool integer(int64_t *v) {
        ws();
        char *end = nullptr;
        long long x = strtoll(p, &end, 10);
        if (end == p) return false;
        p = end;
        *v = x;
        return true;
    }
};

// Parses an object of key -> int (depth 1) into pairs.
bool flat(Reader &r, std::vector<std::pair<std::string, int64_t>> *kv) {
    if (!r.ch('{')) return false;
    if (r.ch('}')) return true;
    do {
        std::string k;
        int64_t v;
        if (!r.str(&k) || !r.ch(':') || !r.integer(&v)) return false;
        kv->push_back({k, v});
    } while (r.ch(','));
    return r.ch('}');
}

}  // namespace

int64_t get(const char *key) {
    std::lock_guard<std::mutex> lk(g_m);
    Knob *k = find(key);
    return k ? k->value : 0;
}

bool known(const char *key) { return find(key) != nullptr; }

std::atomic<uint64_t> g_generation{0};

uint64_t generation() { return g_generation.load(); }

bool set(const char *key, int64_t value) {
    std::lock_guard<std::mutex> lk(g_m);
    Knob *k = find(key);
    if (!k) return false;
    const int64_t v = value < k->lo ? k->lo : (value > k->hi ? k->hi : value);
    if (v != k->value) g_generation.fetch_add(1);
    k->value = v;
    return true;
}

hxc_status load_file(const char *path, int major, int minor) {
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error("tune cache %s: cannot open", path);
        return HXC_E_INVALID;
    }
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    fclose(f);
    Reader r{text.data(), text.data() + text.size()};
    char want[32];
    snprintf(want, sizeof want, "sm_%d%d", major, minor);
    std::vector<std::pair<std::string, int64_t>> kv;
    // nested form: find the object of this architecture
    Reader probe = r;
    bool nested = probe.ch('{') && (probe.ws(), probe.p < probe.e && *probe.p == '"');
    if (nested) {
        std::string k;
        Reader q = probe;
        if (q.str(&k) && q.ch(':') && (q.ws(), q.p < q.e && *q.p == '{')) {
            // {"sm_xy": {...}, ...}
            Reader s = r;
            s.ch('{');
            do {
                std::string arch;
                if (!s.str(&arch) || !s.ch(':')) {
                    set_error("tune cache %s: malformed", path);
                    return HXC_E_INVALID;
                }
                std::vector<std::pair<std::string, int64_t>> one;
                if (!flat(s, &one)) {
                    set_error("tune cache %s: malformed", path);
                    return HXC_E_INVALID;
                }
                if (arch == want) kv = one;
            } while (s.ch(','));
        } else if (!flat(r, &kv)) {
            set_error("tune cache %s: malformed", path);
            return HXC_E_INVALID;
        }
    } else if (!flat(r, &kv)) {
        set_error("tune cache %s: malformed", path);
        return HXC_E_INVALID;
    }
    for (auto &p : kv) set(p.first.c_str(), p.second);  // unknown keys are ignored
    return HXC_OK;
}

void load_default(int major, int minor) {
    static std::once_flag once;
    std::call_once(once, [&] {
        const char *env = getenv("HXC_TUNE_CACHE");
        if (env && *env) {
            load_file(env, major, minor);
            return;
        }
        Dl_info info;
        if (dladdr(reinterpret_cast<void *>(&load_default), &info) && info.dli_fname) {
            std::string p = info.dli_fname;
            size_t slash = p.rfind('/');
            p = (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/tune_cache.json";
            FILE *f = fopen(p.c_str(), "rb");
            if (f) {
                fclose(f);
                load_file(p.c_str(), major, minor);
            }
        }
    });
}

}  // namespace tune
}  // namespace hxc
