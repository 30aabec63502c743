// Autotuner for launch shapes and kernel forms.  A kernel family registers
// candidate launch configurations; the first call with a new key (kernel, mode,
// precision, lattice, nrhs, GPU) times every candidate on the call's own
// operands with CUDA events and keeps the fastest.  Kernels that update their
// operands in place (the SAP block sweeps) are timed in flight instead: the
// sweeps of the first application alternate between the candidate forms.  Choices persist in a small JSON file
// ($LQCD_TUNE_CACHE, default $HOME/.cache/lqcd_tune.json) so later processes
// skip the search.  Kernels whose results do not depend on the launch shape
// (no reductions) are the only ones tuned, so tuning never changes numerics.
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "lqcd_internal.cuh"
#include "lqcd_tune.h"

namespace {

std::mutex g_mu;
std::map<std::string, TuneChoice> g_cache;
bool g_loaded = false;
std::string g_gpu;

std::string cache_path()
{
    const char *p = getenv("LQCD_TUNE_CACHE");
    if (p && *p) return p;
    const char *h = getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/lqcd_tune.json";
}

// file format: {"key": [variant, tx, ty, us, nr, kind], ...} one entry per line
void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    std::ifstream f(cache_path());
    std::string line;
    while (std::getline(f, line)) {
        size_t a = line.find('"'), b = line.find('"', a + 1), l = line.find('['), r = line.find(']');
        if (a == std::string::npos || b == std::string::npos || l == std::string::npos || r == std::string::npos)
            continue;
        std::string key = line.substr(a + 1, b - a - 1);
        std::stringstream ss(line.substr(l + 1, r - l - 1));
        TuneChoice t;
        char comma;
        if (ss >> t.variant >> comma >> t.tx >> comma >> t.ty >> comma >> t.us) {
            if (!(ss >> comma >> t.nr)) t.nr = 1;
            if (!(ss >> comma >> t.kind)) t.kind = 0;
            g_cache[key] = t;
        }
    }
}

void save_locked()
{
    std::string path = cache_path();
    size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        std::string dir = path.substr(0, slash);
        std::string cmd = "mkdir -p '" + dir + "' 2>/dev/null";
        if (system(cmd.c_str()) != 0) return;
    }
    std::string tmp = path + ".tmp";
    std::ofstream f(tmp);
    if (!f) return;
    f << "{\n";
    size_t i = 0;
    for (auto &kv : g_cache) {
        f << "  \"" << kv.first << "\": [" << kv.second.variant << ", " << kv.second.tx << ", " << kv.second.ty
          << ", " << kv.second.us << ", " << kv.second.nr << ", " << kv.second.kind << "]"
          << (++i < g_cache.size() ? "," : "") << "\n";
    }
    f << "}\n";
    f.close();
    std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

std::string tune_key(const lqcd_ctx *c, const char *kernel, int mode, int prec, int nrhs)
{
    if (g_gpu.empty()) {
        cudaDeviceProp p;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) g_gpu = p.name;
        for (auto &ch : g_gpu)
            if (ch == ' ' || ch == '"') ch = '_';
    }
    std::ostringstream s;
    s << kernel << "/m" << mode << "/p" << prec << "/n" << nrhs << "/" << c->g.L[0] << "x" << c->g.L[1] << "x"
      << c->g.L[2] << "x" << c->g.L[3] << "/" << g_gpu;
    return s.str();
}

bool tune_lookup(const std::string &key, TuneChoice *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    *out = it->second;
    return true;
}

void tune_store(const std::string &key, const TuneChoice &t)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    g_cache[key] = t;
    save_locked();
}

bool tune_enabled()
{
    const char *p = getenv("LQCD_TUNE");
    return !(p && p[0] == '0');
}

bool tune_verbose()
{
    const char *p = getenv("LQCD_TUNE_VERBOSE");
    return p && p[0] == '1';
}

// time a launch closure on the context's stream: median of reps
lqcd_status tune_time(lqcd_ctx *c, const std::function<lqcd_status()> &launch, int reps, float *us)
{
    cudaEvent_t e0, e1;
    LQCD_CUDA_CHECK(c, cudaEventCreate(&e0));
    LQCD_CUDA_CHECK(c, cudaEventCreate(&e1));
    LQCD_TRY(launch());   // warm-up (also surfaces launch errors)
    std::vector<float> t;
    for (int i = 0; i < reps; i++) {
        cudaEventRecord(e0, c->stream);
        lqcd_status s = launch();
        cudaEventRecord(e1, c->stream);
        if (s != LQCD_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return s;
        }
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms * 1000.f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    *us = t[t.size() / 2];
    return LQCD_OK;
}

extern "C" LQCD_API lqcd_status lqcd_tune_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.clear();
    g_loaded = false;   // the next lookup reads the cache file again
    return LQCD_OK;
}
