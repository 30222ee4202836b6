// The autotuner's cache: the block parameter s (and, for the batched form, the
// unit size Q of the warp-level schedule) chosen by measurement for a size
// class, kept per device model and persisted as JSON.
//
// Section 5 leaves s (and the thread-block size) as program parameters, and
// the paper's strategy (Section 2.4 with Theorem 1) picks the s that keeps the
// parallelism overhead small while the work stays within a constant factor of
// the optimum; here the candidates the model allows are timed on the device
// and the fastest kept.  A choice is valid for the machine it was measured on,
// so the key holds the device's name and SM count; the size class is a pair of
// log2 buckets (n and m for one product; max_deg + 1 and the batch size for a
// batch) and whether p is at least 2^29 (which changes the fold schedule).
#include <cuda_runtime.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "common.cuh"
#include "tune.cuh"

namespace pm {

namespace {

struct Key {
    std::string device;
    int sms, form, pclass, b1, b2;
    bool operator<(const Key& o) const {
        return std::tie(device, sms, form, pclass, b1, b2) < std::tie(o.device, o.sms, o.form, o.pclass, o.b1, o.b2);
    }
};

std::mutex g_mu;
std::map<Key, TuneChoice> g_cache;
bool g_env_done = false;
std::string g_dev_name[64];
int g_dev_sms[64] = {};

int ilog2(int64_t x) {
    int r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

Key make_key(const std::string& dev, int sms, int form, uint32_t p, int64_t x, int64_t y) {
    if (form == PM_TUNE_PLAIN && x < y) std::swap(x, y);
    return Key{dev, sms, form, p >= (1u << 29) ? 1 : 0, ilog2(x < 1 ? 1 : x), ilog2(y < 1 ? 1 : y)};
}

// The current device's name and SM count (cached per device index); false without a device.
bool identity(std::string* name, int* sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    if (g_dev_sms[dev] == 0) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        g_dev_name[dev] = prop.name;
        g_dev_sms[dev] = prop.multiProcessorCount;
    }
    *name = g_dev_name[dev];
    *sms = g_dev_sms[dev];
    return true;
}

// ---- a small reader for the files tune_save writes ----
struct Reader {
    const char* s;
    size_t i, n;
    void ws() { while (i < n && std::isspace((unsigned char)s[i])) ++i; }
    bool lit(char c) {
        ws();
        if (i < n && s[i] == c) { ++i; return true; }
        return false;
    }
    bool str(std::string* out) {
        ws();
        if (i >= n || s[i] != '"') return false;
        ++i;
        out->clear();
        while (i < n && s[i] != '"') {
            if (s[i] == '\\' && i + 1 < n) ++i;
            out->push_back(s[i++]);
        }
        if (i >= n) return false;
        ++i;
        return true;
    }
    bool num(double* out) {
        ws();
        char* end = nullptr;
        *out = std::strtod(s + i, &end);
        if (end == s + i) return false;
        i = (size_t)(end - s);
        return true;
    }
};

void put_locked(const Key& k, const TuneChoice& v) { g_cache[k] = v; }

pm_status load_locked(const char* path) {
    FILE* f = std::fopen(path, "rb");
    if (!f) return PM_ERR_INVALID_ARG;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    Reader r{text.c_str(), 0, text.size()};
    // {"version": 1, "entries": [ {...}, ... ]}
    std::string key;
    if (!r.lit('{')) return PM_ERR_INVALID_ARG;
    std::map<Key, TuneChoice> found;
    bool have_entries = false;
    while (!r.lit('}')) {
        if (!r.str(&key) || !r.lit(':')) return PM_ERR_INVALID_ARG;
        if (key == "entries") {
            have_entries = true;
            if (!r.lit('[')) return PM_ERR_INVALID_ARG;
            while (!r.lit(']')) {
                if (!r.lit('{')) return PM_ERR_INVALID_ARG;
                Key k{"", 0, 0, 0, 0, 0};
                TuneChoice v{0, 0, -1.0f};
                int seen = 0;
                while (!r.lit('}')) {
                    std::string f2;
                    if (!r.str(&f2) || !r.lit(':')) return PM_ERR_INVALID_ARG;
                    if (f2 == "device") {
                        if (!r.str(&k.device)) return PM_ERR_INVALID_ARG;
                        seen |= 1;
                    } else {
                        double x = 0;
                        if (!r.num(&x)) return PM_ERR_INVALID_ARG;
                        if (f2 == "sms") { k.sms = (int)x; seen |= 2; }
                        else if (f2 == "form") { k.form = (int)x; seen |= 4; }
                        else if (f2 == "p_class") { k.pclass = (int)x; seen |= 8; }
                        else if (f2 == "bucket1") { k.b1 = (int)x; seen |= 16; }
                        else if (f2 == "bucket2") { k.b2 = (int)x; seen |= 32; }
                        else if (f2 == "s") { v.s = (int)x; seen |= 64; }
                        else if (f2 == "q") v.q = (int64_t)x;
                        else if (f2 == "ms") v.ms = (float)x;
                    }
                    r.lit(',');
                }
                if (seen != 127 || (k.form != PM_TUNE_PLAIN && k.form != PM_TUNE_BATCHED)) return PM_ERR_INVALID_ARG;
                found[k] = v;
                r.lit(',');
            }
        } else {  // another field ("version"): a number or a string
            double x;
            std::string sv;
            if (!r.num(&x) && !r.str(&sv)) return PM_ERR_INVALID_ARG;
        }
        r.lit(',');
    }
    if (!have_entries) return PM_ERR_INVALID_ARG;
    for (auto& kv : found) g_cache[kv.first] = kv.second;
    return PM_OK;
}

void env_load_locked() {
    if (g_env_done) return;
    g_env_done = true;
    const char* path = std::getenv("POLYMUL_TUNE_CACHE");
    if (path && *path) load_locked(path);  // a missing or unreadable file leaves the cache empty
}

}  // namespace

bool tune_get(int form, uint32_t p, int64_t x, int64_t y, TuneChoice* out) {
    std::string name;
    int sms = 0;
    if (!identity(&name, &sms)) return false;
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    auto it = g_cache.find(make_key(name, sms, form, p, x, y));
    if (it == g_cache.end()) return false;
    *out = it->second;
    return true;
}

void tune_put(int form, uint32_t p, int64_t x, int64_t y, const TuneChoice& v) {
    std::string name;
    int sms = 0;
    if (!identity(&name, &sms)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    put_locked(make_key(name, sms, form, p, x, y), v);
}

}  // namespace pm

using namespace pm;

extern "C" {

pm_status polymul_tune_save(const char* path) {
    if (!path || !*path) return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return PM_ERR_INVALID_ARG;
    std::fprintf(f, "{\"version\": 1, \"entries\": [");
    bool first = true;
    for (const auto& kv : g_cache) {
        const Key& k = kv.first;
        std::string dev;
        for (char c : k.device) {
            if (c == '"' || c == '\\') dev.push_back('\\');
            dev.push_back(c);
        }
        std::fprintf(f,
                     "%s\n  {\"device\": \"%s\", \"sms\": %d, \"form\": %d, \"p_class\": %d, \"bucket1\": %d, "
                     "\"bucket2\": %d, \"s\": %d, \"q\": %lld, \"ms\": %.6g}",
                     first ? "" : ",", dev.c_str(), k.sms, k.form, k.pclass, k.b1, k.b2, kv.second.s,
                     (long long)kv.second.q, (double)kv.second.ms);
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    const bool ok = std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return PM_ERR_INVALID_ARG;
    }
    return PM_OK;
}

pm_status polymul_tune_load(const char* path) {
    if (!path || !*path) return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    return load_locked(path);
}

pm_status polymul_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_done = true;  // an explicit clear also drops what the environment named
    g_cache.clear();
    return PM_OK;
}

pm_status polymul_tune_lookup(const char* device, int sms, int form, uint32_t p, int64_t x, int64_t y, int* s,
                              int64_t* q) {
    if (!device || !s || !q || (form != PM_TUNE_PLAIN && form != PM_TUNE_BATCHED)) return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    auto it = g_cache.find(make_key(device, sms, form, p, x, y));
    *s = it == g_cache.end() ? 0 : it->second.s;
    *q = it == g_cache.end() ? 0 : it->second.q;
    return PM_OK;
}

}  // extern "C"
