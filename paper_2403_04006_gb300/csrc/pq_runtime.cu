// pq_runtime.cu -- runtime services of the library that are not kernels:
// device allocations (counted, with a test hook that makes one fail), the
// process-wide tuning table of chunk lengths per photon number, and its JSON
// cache on disk.
#include <cuda_runtime.h>

#include <atomic>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pq.h"
#include "pq_kernels.h"

namespace pqi {

// ---------------------------------------------------------------- allocations
static std::atomic<int64_t> g_live_device{0};
static std::atomic<int64_t> g_live_host{0};
static std::mutex g_fail_mu;
static int64_t g_fail_after = -1;  // < 0: disarmed

// True if the test hook says that this allocation is the one that fails.
static bool hook_fails()
{
    std::lock_guard<std::mutex> lk(g_fail_mu);
    if (g_fail_after < 0)
        return false;
    if (g_fail_after == 0) {
        g_fail_after = -1;  // one-shot
        return true;
    }
    --g_fail_after;
    return false;
}

cudaError_t dev_alloc(void** p, size_t bytes)
{
    *p = nullptr;
    if (hook_fails())
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        g_live_device.fetch_add(1);
    } else {
        *p = nullptr;
        cudaGetLastError();  // the failure is reported here, not by a later launch check
    }
    return e;
}

void dev_free(void* p)
{
    if (!p)
        return;
    cudaFree(p);
    g_live_device.fetch_sub(1);
}

bool host_object_alloc_ok()
{
    if (hook_fails())
        return false;
    g_live_host.fetch_add(1);
    return true;
}

void host_object_freed() { g_live_host.fetch_sub(1); }

// ---------------------------------------------------------------- tuning table
static std::mutex g_tune_mu;
static int32_t g_tune[PQ_MAX_N + 1] = {0};

int tune_get(int n)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (n < 0 || n > PQ_MAX_N) ? 0 : g_tune[n];
}

void tune_set(int n, int v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (n >= 0 && n <= PQ_MAX_N)
        g_tune[n] = v;
}

// ---------------------------------------------------------------- JSON cache
// The cache file is one JSON object:
//   {"format": "pq-gb300 tuning table", "tables": {"<device key>": [49 ints], ...}}
// with entry n of a table the chunk log2 for permanents of n photons (0: the
// default).  The reader below accepts any JSON; it keeps the "tables" member
// and ignores everything else.
struct JsonReader {
    const char* s;
    const char* e;
    bool ok = true;

    void ws()
    {
        while (s < e && std::isspace((unsigned char)*s))
            ++s;
    }
    bool eat(char c)
    {
        ws();
        if (s < e && *s == c) {
            ++s;
            return true;
        }
        return false;
    }
    bool str(std::string& out)
    {
        ws();
        if (s >= e || *s != '"')
            return ok = false;
        ++s;
        out.clear();
        while (s < e && *s != '"') {
            if (*s == '\\') {
                ++s;
                if (s >= e)
                    return ok = false;
                switch (*s) {
                case 'n': out += '\n'; break;
                case 't': out += '\t'; break;
                case 'u':  // keep the escape as text; keys written here never use it
                    out += "\\u";
                    break;
                default: out += *s;
                }
                ++s;
                continue;
            }
            out += *s++;
        }
        if (s >= e)
            return ok = false;
        ++s;
        return true;
    }
    bool number(double& v)
    {
        ws();
        char* end = nullptr;
        v = std::strtod(s, &end);
        if (end == s)
            return ok = false;
        s = end;
        return true;
    }
    // Skip one value of any kind.
    bool skip()
    {
        ws();
        if (s >= e)
            return ok = false;
        if (*s == '"') {
            std::string t;
            return str(t);
        }
        if (*s == '{' || *s == '[') {
            const char close = (*s == '{') ? '}' : ']';
            const bool obj = (*s == '{');
            ++s;
            if (eat(close))
                return true;
            do {
                if (obj) {
                    std::string k;
                    if (!str(k) || !eat(':'))
                        return ok = false;
                }
                if (!skip())
                    return false;
            } while (eat(','));
            return eat(close) || (ok = false);
        }
        for (const char* w : {"true", "false", "null"}) {
            const size_t n = std::strlen(w);
            if ((size_t)(e - s) >= n && std::strncmp(s, w, n) == 0) {
                s += n;
                return true;
            }
        }
        double v;
        return number(v);
    }
    bool int_array(std::vector<int32_t>& out)
    {
        out.clear();
        if (!eat('['))
            return ok = false;
        if (eat(']'))
            return true;
        do {
            double v;
            if (!number(v))
                return false;
            if (!(v >= -2147483648.0 && v <= 2147483647.0))  // also rejects NaN
                return ok = false;
            out.push_back((int32_t)v);
        } while (eat(','));
        return eat(']') || (ok = false);
    }
};

using Tables = std::map<std::string, std::vector<int32_t>>;

// Read the tables of a cache file.  A missing file gives no tables and true;
// a malformed one gives false.
static bool read_tables(const char* path, Tables& tables)
{
    tables.clear();
    FILE* f = std::fopen(path, "rb");
    if (!f)
        return true;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0)
        text.append(buf, got);
    std::fclose(f);
    JsonReader r{text.data(), text.data() + text.size()};
    if (!r.eat('{'))
        return false;
    if (r.eat('}'))
        return true;
    do {
        std::string key;
        if (!r.str(key) || !r.eat(':'))
            return false;
        if (key == "tables") {
            if (!r.eat('{'))
                return false;
            if (r.eat('}'))
                continue;
            do {
                std::string dev;
                std::vector<int32_t> t;
                if (!r.str(dev) || !r.eat(':') || !r.int_array(t))
                    return false;
                tables[dev] = t;
            } while (r.eat(','));
            if (!r.eat('}'))
                return false;
        } else if (!r.skip()) {
            return false;
        }
    } while (r.eat(','));
    return r.eat('}') && r.ok;
}

static std::string json_escape(const std::string& k)
{
    std::string o;
    for (char c : k) {
        if (c == '"' || c == '\\')
            o += '\\';
        if ((unsigned char)c < 0x20)
            continue;
        o += c;
    }
    return o;
}

static bool write_tables(const char* path, const Tables& tables)
{
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f)
        return false;
    std::fprintf(f, "{\"format\": \"pq-gb300 tuning table\", \"tables\": {");
    bool first = true;
    for (const auto& kv : tables) {
        std::fprintf(f, "%s\n  \"%s\": [", first ? "" : ",", json_escape(kv.first).c_str());
        for (size_t i = 0; i < kv.second.size(); ++i)
            std::fprintf(f, "%s%d", i ? ", " : "", kv.second[i]);
        std::fprintf(f, "]");
        first = false;
    }
    std::fprintf(f, "\n}}\n");
    const bool good = std::fflush(f) == 0;
    std::fclose(f);
    if (!good || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

// "<device name> (<SMs> SMs)" of the current device.
static int current_device_key(std::string& key)
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return report(PQ_ERR_CUDA, "no CUDA device to name the tuning table: pass a key");
    key = std::string(prop.name) + " (" + std::to_string(prop.multiProcessorCount) + " SMs)";
    return PQ_OK;
}

}  // namespace pqi

using namespace pqi;

extern "C" int pq_debug_fail_allocation(int64_t after)
{
    std::lock_guard<std::mutex> lk(g_fail_mu);
    g_fail_after = after < 0 ? -1 : after;
    return PQ_OK;
}

extern "C" int pq_debug_live_allocations(int64_t* device_buffers, int64_t* host_objects)
{
    if (!device_buffers || !host_objects)
        return report(PQ_ERR_ARG, "null argument");
    *device_buffers = g_live_device.load();
    *host_objects = g_live_host.load();
    return PQ_OK;
}

extern "C" int pq_tune_table_get(int32_t* log2)
{
    if (!log2)
        return report(PQ_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::memcpy(log2, g_tune, sizeof(g_tune));
    return PQ_OK;
}

extern "C" int pq_tune_table_set(const int32_t* log2)
{
    if (!log2)
        return report(PQ_ERR_ARG, "null argument");
    for (int n = 0; n <= PQ_MAX_N; ++n)
        if (log2[n] < 0 || log2[n] > 30)
            return report(PQ_ERR_ARG, "tuning entry outside [0, 30]");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::memcpy(g_tune, log2, sizeof(g_tune));
    return PQ_OK;
}

extern "C" int pq_tune_cache_save(const char* path, const char* device_key)
{
    if (!path)
        return report(PQ_ERR_ARG, "null path");
    std::string key = device_key ? device_key : "";
    if (!device_key) {
        int rc = current_device_key(key);
        if (rc != PQ_OK)
            return rc;
    }
    Tables tables;
    if (!read_tables(path, tables))
        return report(PQ_ERR_ARG, "tuning cache exists but is not a readable tuning table");
    std::vector<int32_t> t(PQ_MAX_N + 1);
    pq_tune_table_get(t.data());
    tables[key] = t;
    if (!write_tables(path, tables))
        return report(PQ_ERR_ARG, "cannot write the tuning cache");
    return PQ_OK;
}

extern "C" int pq_tune_cache_load(const char* path, const char* device_key, int32_t* found)
{
    if (!path || !found)
        return report(PQ_ERR_ARG, "null argument");
    *found = 0;
    std::string key = device_key ? device_key : "";
    if (!device_key) {
        int rc = current_device_key(key);
        if (rc != PQ_OK)
            return rc;
    }
    Tables tables;
    if (!read_tables(path, tables))
        return report(PQ_ERR_ARG, "tuning cache is not a readable tuning table");
    auto it = tables.find(key);
    if (it == tables.end())
        return PQ_OK;
    if (it->second.size() != (size_t)(PQ_MAX_N + 1))
        return report(PQ_ERR_ARG, "tuning table of the wrong length");
    int rc = pq_tune_table_set(it->second.data());
    if (rc == PQ_OK)
        *found = 1;
    return rc;
}
