// Autotuner of the spectral-energy tile shape (BT x BX x BY outputs per CTA).  Candidates
// are timed with CUDA events on the caller's stream; the fastest shape is cached per
// (cube side L, precision, size class) for the process, and the cache can be saved to and
// loaded from a small text file.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "sal_internal.cuh"

namespace sal {

namespace {

constexpr int kClasses = 2;                    // 0: fewer than 16 M voxels per volume, 1: larger
struct Entry {
    int shape;
    float ms;
    bool set;
};
std::mutex g_mu;
Entry g_cache[kMaxL + 1][3][kClasses];

bool valid_key(int L, int precision, int cls)
{
    return L >= 3 && L <= kMaxL && (L & 1) && precision >= 0 && precision < 3 && cls >= 0 && cls < kClasses;
}

}  // namespace

int size_class_of(int64_t n_vox) { return n_vox < (int64_t)16 << 20 ? 0 : 1; }

int autotune_lookup(int L, int precision, int cls)
{
    if (!valid_key(L, precision, cls)) return 0;
    std::lock_guard<std::mutex> lock(g_mu);
    const Entry &e = g_cache[L][precision][cls];
    return e.set ? e.shape : 0;
}

bool autotune_get_ms(int L, int precision, int cls, float *ms)
{
    *ms = 0.f;
    if (!valid_key(L, precision, cls)) return false;
    std::lock_guard<std::mutex> lock(g_mu);
    const Entry &e = g_cache[L][precision][cls];
    if (e.set) *ms = e.ms;
    return e.set;
}

void autotune_store(int L, int precision, int cls, int shape, float ms)
{
    if (!valid_key(L, precision, cls)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[L][precision][cls] = Entry{shape, ms, true};
}

void autotune_clear()
{
    std::lock_guard<std::mutex> lock(g_mu);
    memset(g_cache, 0, sizeof(g_cache));
}

cudaError_t autotune_run(const EVolDesc *vols, int n, int L, int bnd, int precision, cudaStream_t s, int *best,
                         float *best_ms)
{
    const int ns = energy_num_shapes(L);
    if (ns <= 0 || n < 1) return cudaErrorInvalidValue;
    int64_t nmax = 0;
    for (int i = 0; i < n; ++i) nmax = vols[i].T * vols[i].X * vols[i].Y > nmax ? vols[i].T * vols[i].X * vols[i].Y : nmax;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    int arg = 0;
    float argms = 0.f;
    for (int k = 0; k < ns && e == cudaSuccess; ++k) {
        e = launch_energy_fp32_batch(vols, n, L, bnd, k, n > 1, s);                 // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_energy_fp32_batch(vols, n, L, bnd, k, n > 1, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (e == cudaSuccess && (k == 0 || ms < argms)) {
            arg = k;
            argms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    autotune_store(L, precision, size_class_of(nmax), arg, argms);
    *best = arg;
    *best_ms = argms;
    return cudaSuccess;
}

// Text format, one entry per line: "L precision size_class shape milliseconds".
int autotune_save(const char *path)
{
    FILE *f = fopen(path, "w");
    if (!f) return -1;
    std::lock_guard<std::mutex> lock(g_mu);
    fprintf(f, "# sal autotune cache v1: L precision size_class shape ms\n");
    for (int L = 3; L <= kMaxL; L += 2)
        for (int p = 0; p < 3; ++p)
            for (int c = 0; c < kClasses; ++c)
                if (g_cache[L][p][c].set) fprintf(f, "%d %d %d %d %.6f\n", L, p, c, g_cache[L][p][c].shape, g_cache[L][p][c].ms);
    return fclose(f) == 0 ? 0 : -1;
}

// Every line is validated before anything is stored: a malformed file changes nothing.
int autotune_load(const char *path)
{
    FILE *f = fopen(path, "r");
    if (!f) return -1;
    Entry fresh[kMaxL + 1][3][kClasses];
    memset(fresh, 0, sizeof(fresh));
    char line[256];
    int rc = 0, lines = 0;
    if (!fgets(line, sizeof(line), f) || strncmp(line, "# sal autotune cache v1", 23) != 0) rc = -2;
    while (rc == 0 && fgets(line, sizeof(line), f)) {
        int L, p, c, sh;
        float ms;
        char extra[8];
        if (line[0] == '\n') continue;
        if (sscanf(line, "%d %d %d %d %f %7s", &L, &p, &c, &sh, &ms, extra) != 5 || !valid_key(L, p, c) || sh < 0 ||
            sh >= energy_num_shapes(L) || !(ms >= 0.f)) {
            rc = -3;
            break;
        }
        fresh[L][p][c] = Entry{sh, ms, true};
        ++lines;
    }
    fclose(f);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    memcpy(g_cache, fresh, sizeof(g_cache));
    return lines;
}

}  // namespace sal
