// Hopping-term launches: grid assignment, the plain and xpay instantiations
// of the kernel templates in dslash_kernel.cuh, and the launch-shape
// autotuner.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "dslash_kernel.cuh"

namespace cola {

// Site blocks per lattice for block_x (each repeated for the ngroups
// right-hand-side groups); returns the grid size.
static int assign_blocks(DslashArgs &A, int bx) {
    int total = 0;
    for (int l = 0; l < A.nlat; ++l) {
        A.lat[l].block0 = total;
        A.lat[l].nblocks = (A.lat[l].g.Vh + bx - 1) / bx;
        total += A.lat[l].nblocks * A.ngroups;
    }
    return total;
}

static cudaError_t launch_now(int prec, int recon, DslashArgs &A, int nparity, bool dagger, int epi, int block_x,
                              cudaStream_t s) {
    if (A.rhs_per_thread < 1) A.rhs_per_thread = 1;
    if (!mrhs_supported(prec, A.rhs_per_thread) || (A.rhs_per_thread > 1 && staged_depth(prec) > 0))
        return cudaErrorInvalidValue;
    const int per_group = A.rhs_per_block * A.rhs_per_thread;
    A.ngroups = (A.nrhs + per_group - 1) / per_group;
    const int nb = assign_blocks(A, block_x);
    if (epi == EPI_CLOVER_X || epi == EPI_CLOVER_INV)
        return launch_dslash_clover(prec, recon, A, nparity, dagger, epi, block_x, nb, s);
    return launch_pr<EPI_HOP, EPI_XPAY>(prec, recon, A, nparity, dagger, epi, block_x, nb, s);
}

// ---------------------------------------------------------------- autotune --
// Launch shape (threads per block along sites, right-hand sides per block)
// chosen per configuration by timing the candidates on the caller's stream
// the first time a configuration is seen outside stream capture.  The
// timed launches write only `out` (never an input), without the fused
// reduction or solver-state filtering, so tuning changes no result.  Entries
// are kept per process and, with COLA_TUNE_CACHE=<file>, in that file.
// COLA_TUNE=0 disables tuning (defaults are used).
struct TuneEntry {
    int bx, by, nr;  // sites per block, right-hand sides per block (threads), right-hand sides per thread
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneEntry> g_tune;
static bool g_tune_loaded = false;

static std::string tune_key(int prec, int recon, const DslashArgs &A, int nparity, bool dagger, int epi) {
    std::string k = "dslash p" + std::to_string(prec) + " r" + std::to_string(recon) + " d" + std::to_string(dagger) +
                    " e" + std::to_string(epi) + " np" + std::to_string(nparity) + " n" + std::to_string(A.nrhs) +
                    " s" + std::to_string(staged_depth(prec));
    for (int l = 0; l < A.nlat; ++l) {
        const Geom &g = A.lat[l].g;
        k += " " + std::to_string(g.L[0]) + "x" + std::to_string(g.L[1]) + "x" + std::to_string(g.L[2]) + "x" +
             std::to_string(g.L[3]);
    }
    return k;
}

static void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("COLA_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
        char *bar = strrchr(line, '|');
        if (!bar) continue;
        int bx = 0, by = 0, nr = 1;
        const int n = sscanf(bar + 1, "%d %d %d", &bx, &by, &nr);
        if (n < 2 || bx < 32 || by < 1 || nr < 1) continue;
        *bar = 0;
        g_tune[std::string(line)] = {bx, by, n == 3 ? nr : 1};
    }
    fclose(f);
}

static void tune_store_locked(const std::string &key, TuneEntry e) {
    g_tune[key] = e;
    const char *path = getenv("COLA_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s|%d %d %d\n", key.c_str(), e.bx, e.by, e.nr);
    fclose(f);
}

static bool tuning_enabled() {
    static const bool on = [] {
        const char *e = getenv("COLA_TUNE");
        return !(e && e[0] == '0');
    }();
    return on;
}

// While a TuneOnlyScope is alive on this thread, launch_dslash tunes unseen
// configurations and launches nothing else.
static thread_local int g_tune_only = 0;
TuneOnlyScope::TuneOnlyScope() { ++g_tune_only; }
TuneOnlyScope::~TuneOnlyScope() { --g_tune_only; }

// True if the launch's tuning runs could change an input.  A single-parity
// launch writes only parity p of out and reads parity 1 - p of in, so out ==
// in (one field holding two temporaries in its two parity halves) is no
// alias there; the xpay input is read at parity p and always is one.
static bool outputs_alias_inputs(const DslashArgs &A, int nparity) {
    for (int l = 0; l < A.nlat; ++l) {
        if (A.lat[l].out == A.lat[l].xin) return true;
        if (A.lat[l].out == A.lat[l].in && nparity != 1) return true;
    }
    return false;
}

static TuneEntry tune(int prec, int recon, const DslashArgs &A0, int nparity, bool dagger, int epi,
                      cudaStream_t s) {
    TuneEntry best = {default_dslash_block(prec, A0.rhs_per_block), A0.rhs_per_block, 1};
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return best;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return best;
    }
    const int bys[] = {1, 2, 4, 8};
    const int bxs[] = {32, 64, 128, 256};
    const int nrs[] = {1, 2, 4};
    const bool staged = prec != COLA_F64 && staged_depth(prec) > 0;
    for (int nr : nrs) {
    if (!mrhs_supported(prec, nr) || (nr > 1 && staged) || nr > A0.nrhs) continue;
    for (int by : bys) {
        if (by * nr > A0.nrhs && by > 1) continue;
        for (int bx : bxs) {
            if (bx * by > 256 || bx * by < 64) continue;
            if (staged && bx * by != kStagedThreads) continue;
            DslashArgs A = A0;
            A.rhs_per_block = by;
            A.rhs_per_thread = nr;
            A.state = nullptr;
            A.filter_ru = 0;
            A.red = nullptr;
            bool ok = launch_now(prec, recon, A, nparity, dagger, epi, bx, s) == cudaSuccess;
            ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
            for (int r = 0; r < 3 && ok; ++r) ok = launch_now(prec, recon, A, nparity, dagger, epi, bx, s) == cudaSuccess;
            ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.f;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best = {bx, by, nr};
            }
            cudaGetLastError();
        }
    }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

cudaError_t launch_dslash(int prec, int recon, DslashArgs &A, int nparity, bool dagger, int epi, int block_x,
                          cudaStream_t s) {
    if (A.nlat < 1 || A.nlat > kMaxBatch) return cudaErrorInvalidValue;
    if (block_x <= 0) {
        block_x = default_dslash_block(prec, A.rhs_per_block);
        if (tuning_enabled()) {
            const std::string key = tune_key(prec, recon, A, nparity, dagger, epi);
            std::lock_guard<std::mutex> lock(g_tune_mu);
            tune_load_locked();
            auto it = g_tune.find(key);
            if (it == g_tune.end()) {
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
                    !outputs_alias_inputs(A, nparity)) {
                    tune_store_locked(key, tune(prec, recon, A, nparity, dagger, epi, s));
                    it = g_tune.find(key);
                }
            }
            if (it != g_tune.end()) {
                block_x = it->second.bx;
                A.rhs_per_block = it->second.by;
                A.rhs_per_thread = it->second.nr;
            }
        }
    }
    if (g_tune_only) return cudaSuccess;
    // COLA_DSLASH_NR=n forces n right-hand sides per thread where the kernel
    // supports it (tests of the multi-right-hand-side kernel)
    static const int env_nr = [] {
        const char *e = getenv("COLA_DSLASH_NR");
        return e ? atoi(e) : 0;
    }();
    if (env_nr > 0 && mrhs_supported(prec, env_nr) && staged_depth(prec) == 0 && A.nrhs > 1) {
        A.rhs_per_thread = env_nr;
        if (A.rhs_per_block * env_nr > A.nrhs) A.rhs_per_block = 1;
    }
    if (prec != COLA_F64 && staged_depth(prec) > 0 && block_x * A.rhs_per_block != kStagedThreads) {
        // the staged kernel's shared-memory layout is built for kStagedThreads threads
        A.rhs_per_block = std::min(A.rhs_per_block, 4);
        block_x = kStagedThreads / A.rhs_per_block;
    }
    return launch_now(prec, recon, A, nparity, dagger, epi, block_x, s);
}

// Threads per block along the sites; COLA_DSLASH_BLOCK overrides (tuning runs).
int default_dslash_block(int prec, int rhs_per_block) {
    static const int env_bx = [] {
        const char *e = getenv("COLA_DSLASH_BLOCK");
        int v = e ? atoi(e) : 0;
        return (v >= 32 && v <= 1024 && v % 32 == 0) ? v : 0;
    }();
    int bx = env_bx ? env_bx : 128;
    while (bx * rhs_per_block > 256 && bx > 32) bx >>= 1;
    return bx;
}

}  // namespace cola
