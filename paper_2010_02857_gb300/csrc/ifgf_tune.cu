// Persistent tune cache of the batched path's tile shapes.
//
// ifgf_plan_autotune times the candidate tile shapes on a plan (a few evaluations'
// worth of device time).  A later plan of the same workload on the same kind of device
// takes the same shapes, so the choice is kept in a text file, one line per workload:
//
//     <key> <leaf shape> <cone CTAs per SM>
//
// The key names the device (its name and SM count), the plan's precision and
// interpolation order, the right-hand-side count, and the sizes that decide how the
// work splits: the point count, the depth, the leaf factor count and the rows of the
// cone contraction (cousin plus upward evaluations).  Lines are appended whole; the
// last valid line for a key wins and malformed lines are skipped, so the file may be
// shared by processes and edited by hand.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "ifgf_internal.h"

namespace {

constexpr int kMaxKey = 480;  // bytes of a key, without the terminating zero
constexpr int kMaxLine = 1024;

bool key_ok(const char *key)
{
    if (!key) return false;
    const size_t n = strlen(key);
    if (n == 0 || n > (size_t)kMaxKey) return false;
    for (size_t i = 0; i < n; ++i)
        if (key[i] <= ' ' || key[i] == 127) return false;  // one whitespace-free token
    return true;
}

bool choice_ok(int leaf, int ctas) { return leaf >= 0 && leaf <= 2 && ctas >= 1 && ctas <= 2; }

}  // namespace

extern "C" ifgf_status ifgf_tune_cache_lookup(const char *path, const char *key, int *found, int *choice)
{
    if (!path || !found || !choice || !key_ok(key)) return IFGF_EINVAL;
    *found = 0;
    FILE *f = fopen(path, "r");
    if (!f) return IFGF_OK;  // no file yet: nothing cached
    char line[kMaxLine];
    char k[kMaxLine];
    while (fgets(line, sizeof line, f)) {
        const size_t len = strlen(line);
        if (len + 1 == sizeof line && line[len - 1] != '\n') {
            // an over-long line: skip the rest of it, it cannot hold a valid entry
            int c;
            while ((c = fgetc(f)) != EOF && c != '\n') {
            }
            continue;
        }
        int leaf = -1, ctas = -1;
        char extra[2];
        if (sscanf(line, "%1023s %d %d %1s", k, &leaf, &ctas, extra) != 3) continue;
        if (strcmp(k, key) != 0 || !choice_ok(leaf, ctas)) continue;
        choice[0] = leaf;
        choice[1] = ctas;
        *found = 1;  // keep reading: a later line for the key replaces this one
    }
    fclose(f);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_tune_cache_store(const char *path, const char *key, const int *choice)
{
    if (!path || !choice || !key_ok(key) || !choice_ok(choice[0], choice[1])) return IFGF_EINVAL;
    char line[kMaxLine];
    const int n = snprintf(line, sizeof line, "%s %d %d\n", key, choice[0], choice[1]);
    if (n <= 0 || n >= (int)sizeof line) return IFGF_EINVAL;
    FILE *f = fopen(path, "a");
    if (!f) return IFGF_EINVAL;
    // one write of the whole line, so that appends of several processes do not interleave
    setvbuf(f, nullptr, _IOFBF, sizeof line);
    const bool ok = fwrite(line, 1, (size_t)n, f) == (size_t)n;
    const bool closed = fclose(f) == 0;
    return ok && closed ? IFGF_OK : IFGF_EINVAL;
}

extern "C" ifgf_status ifgf_plan_tune_key(const ifgf_plan *plan, int nrhs, char *buf, int cap)
{
    if (!plan || !buf || cap <= 0) return IFGF_EINVAL;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, plan->device) != cudaSuccess) {
        cudaGetLastError();
        return IFGF_ECUDA;
    }
    std::string name(prop.name);
    for (char &c : name)
        if (c <= ' ' || c == 127) c = '_';
    long long rows = 0;
    for (int d = 1; d <= plan->D; ++d) rows += plan->lh[d].cousin_evals + plan->lh[d].upward_evals;
    char key[kMaxLine];
    const int n = snprintf(key, sizeof key, "%s/sm%d/cc%d.%d;prec%d;order%dx%d;nrhs%d;n%lld;D%d;leaf%lld;rows%lld",
                           name.c_str(), prop.multiProcessorCount, prop.major, prop.minor, plan->precision,
                           plan->Ps, plan->Pang, nrhs, (long long)plan->n, plan->D, (long long)plan->leaf_evals,
                           rows);
    if (n <= 0 || n > kMaxKey || !key_ok(key) || n + 1 > cap) return IFGF_EINVAL;
    memcpy(buf, key, (size_t)n + 1);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_autotune_cached(ifgf_plan *plan, int nrhs, int reps, const char *path, int *choice,
                                                 int *hit, void *stream)
{
    if (!plan || !path || !hit) return IFGF_EINVAL;
    *hit = 0;
    char key[kMaxKey + 1];
    ifgf_status s = ifgf_plan_tune_key(plan, nrhs, key, sizeof key);
    if (s != IFGF_OK) {
        plan->last_error = "autotune: forming the tune-cache key";
        return s;
    }
    int c[2] = {0, 2}, found = 0;
    s = ifgf_tune_cache_lookup(path, key, &found, c);
    if (s != IFGF_OK) return s;
    if (found) {
        // the same checks as a tuning run, so that a cached entry is used only where one
        // could have been made
        if (!ifgf_is_batched(plan->precision) || nrhs < 2 || nrhs % 2 || nrhs > ifgf_batched_max_nrhs(plan->Ps) ||
            nrhs > plan->max_nrhs || reps < 1) {
            plan->last_error = "autotune: batched plan, even nrhs in [2, min(64, max_nrhs)] and reps >= 1";
            return IFGF_EINVAL;
        }
        s = ifgf_plan_set_tiles(plan, c[0], c[1]);
        if (s != IFGF_OK) return s;
        *hit = 1;
    } else {
        s = ifgf_plan_autotune(plan, nrhs, reps, nullptr, c, stream);
        if (s != IFGF_OK) return s;
        if (ifgf_tune_cache_store(path, key, c) != IFGF_OK) {
            plan->last_error = std::string("autotune: cannot append to the tune cache ") + path;
            return IFGF_EINVAL;
        }
    }
    if (choice) {
        choice[0] = c[0];
        choice[1] = c[1];
    }
    return IFGF_OK;
}
