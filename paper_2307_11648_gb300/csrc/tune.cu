// Autotuning of launch shapes (host code).
//
// The handle keeps a small table of tuned choices, each keyed by what is tuned and a bucket of
// the problem's sizes; kernels look their choice up at launch and fall back to a built-in
// default.  Tuned now: the size-class split of the FP64 fill (groups of at most `split`
// members run in the 4-worker launch, larger ones in the large-group launch, each with its
// own shared-memory layout and occupancy) and the large-group launch's worker warps (8 or
// 12); and the supernodal selection's launch plan (sic_tune_select_aggregated in
// select_aggregated.cu: threads per CTA, state in shared memory or in the workspace).  sic_tune_build_factor times every candidate split on the caller's own problem with
// CUDA events, then the worker count at the best split, and keeps the fastest; sic_tune_save and
// sic_tune_load keep the table in a text file, one "op a b value ms" line per entry.
#include <stdio.h>

#include "sic_internal.cuh"

int tune_get(const sic_handle* h, int op, int a, int b, int fallback) {
    if (!h) return fallback;
    for (int i = 0; i < h->n_tune; ++i)
        if (h->tune[i].op == op && h->tune[i].a == a && h->tune[i].b == b) return h->tune[i].value;
    return fallback;
}

void tune_put(sic_handle* h, int op, int a, int b, int value, float ms) {
    for (int i = 0; i < h->n_tune; ++i)
        if (h->tune[i].op == op && h->tune[i].a == a && h->tune[i].b == b) {
            h->tune[i].value = value;
            h->tune[i].ms = ms;
            return;
        }
    if (h->n_tune >= TUNE_MAX) return;  // table full: the call keeps its default
    h->tune[h->n_tune++] = TuneEntry{op, a, b, value, ms};
}

extern "C" sic_status sic_tune_build_factor(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                            const int64_t* grp_ptr, int64_t n_grp, int32_t max_m,
                                            const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                                            const int64_t* col_ptr, int32_t* row_idx, double* val, double* logv,
                                            double* sum_logv, void* ws, size_t ws_bytes, void* stream,
                                            int32_t* best_split) {
    if (!h) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int cands[] = {8, 12, 16, 20, 24, 28, 32, 40, 48, 64};
    cudaEvent_t e0, e1;
    SIC_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SIC_ERR_CUDA;
    }
    sic_status st = SIC_OK;
    int best = -1, last = 0;
    float best_ms = 0.f;
    for (int ci = 0; ci < (int)(sizeof(cands) / sizeof(cands[0])) && st == SIC_OK; ++ci) {
        const int split = cands[ci] < max_m ? cands[ci] : max_m;
        if (split == last) break;  // ascending candidates: once capped at max_m, every one is tried
        last = split;
        tune_put(h, TUNE_FILL_SPLIT, k, max_m, split, 0.f);
        float ms = 0.f;
        for (int rep = 0; rep < 3 && st == SIC_OK; ++rep) {  // the first run warms up
            if (cudaEventRecord(e0, s) != cudaSuccess) st = SIC_ERR_CUDA;
            if (st == SIC_OK)
                st = sic_build_factor(h, pts, n, kp, grp_ptr, n_grp, max_m, sel_idx, sel_count, k, col_ptr, row_idx,
                                      val, logv, sum_logv, ws, ws_bytes, stream);
            if (st == SIC_OK && cudaEventRecord(e1, s) != cudaSuccess) st = SIC_ERR_CUDA;
            if (st == SIC_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SIC_ERR_CUDA;
            float t = 0.f;
            if (st == SIC_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = SIC_ERR_CUDA;
            if (rep == 1 || (rep > 1 && t < ms)) ms = t;
        }
        if (st == SIC_OK && (best < 0 || ms < best_ms)) {
            best = split;
            best_ms = ms;
        }
    }
    // then the worker count of the large-group launch at that split
    int best_nt = 256;
    if (st == SIC_OK && best < max_m) {
        tune_put(h, TUNE_FILL_SPLIT, k, max_m, best, best_ms);
        tune_put(h, TUNE_FILL_BIGNT, k, max_m, 384, 0.f);
        float ms = 0.f;
        for (int rep = 0; rep < 3 && st == SIC_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) st = SIC_ERR_CUDA;
            if (st == SIC_OK)
                st = sic_build_factor(h, pts, n, kp, grp_ptr, n_grp, max_m, sel_idx, sel_count, k, col_ptr, row_idx,
                                      val, logv, sum_logv, ws, ws_bytes, stream);
            if (st == SIC_OK && cudaEventRecord(e1, s) != cudaSuccess) st = SIC_ERR_CUDA;
            if (st == SIC_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SIC_ERR_CUDA;
            float t = 0.f;
            if (st == SIC_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = SIC_ERR_CUDA;
            if (rep == 1 || (rep > 1 && t < ms)) ms = t;
        }
        if (st == SIC_OK && ms < best_ms) {
            best_nt = 384;
            best_ms = ms;
        }
    }
    if (st == SIC_OK) {
        tune_put(h, TUNE_FILL_SPLIT, k, max_m, best, best_ms);
        tune_put(h, TUNE_FILL_BIGNT, k, max_m, best_nt, best_ms);
        // leave the outputs of the chosen configuration (identical for every split)
        st = sic_build_factor(h, pts, n, kp, grp_ptr, n_grp, max_m, sel_idx, sel_count, k, col_ptr, row_idx, val,
                              logv, sum_logv, ws, ws_bytes, stream);
        if (best_split) *best_split = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

extern "C" int32_t sic_tune_count(const sic_handle* h) { return h ? h->n_tune : 0; }

extern "C" sic_status sic_tune_entry(const sic_handle* h, int32_t i, int32_t* op, int32_t* a, int32_t* b,
                                     int32_t* value, float* ms) {
    if (!h || i < 0 || i >= h->n_tune || !op || !a || !b || !value || !ms) return SIC_ERR_INVALID;
    *op = h->tune[i].op;
    *a = h->tune[i].a;
    *b = h->tune[i].b;
    *value = h->tune[i].value;
    *ms = h->tune[i].ms;
    return SIC_OK;
}

extern "C" sic_status sic_tune_save(const sic_handle* h, const char* path) {
    if (!h || !path) return SIC_ERR_INVALID;
    FILE* f = fopen(path, "w");
    if (!f) return SIC_ERR_INVALID;
    fprintf(f, "# libsic tuned launch choices: op a b value ms\n");
    for (int i = 0; i < h->n_tune; ++i)
        fprintf(f, "%d %d %d %d %.6f\n", h->tune[i].op, h->tune[i].a, h->tune[i].b, h->tune[i].value,
                (double)h->tune[i].ms);
    const int bad = ferror(f);
    fclose(f);
    return bad ? SIC_ERR_INVALID : SIC_OK;
}

extern "C" sic_status sic_tune_load(sic_handle* h, const char* path) {
    if (!h || !path) return SIC_ERR_INVALID;
    FILE* f = fopen(path, "r");
    if (!f) return SIC_ERR_INVALID;
    char line[256];
    sic_status st = SIC_OK;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int op, a, b, value;
        double ms;
        if (sscanf(line, "%d %d %d %d %lf", &op, &a, &b, &value, &ms) != 5 ||
            (op != TUNE_FILL_SPLIT && op != TUNE_FILL_BIGNT && op != TUNE_SELECT_AGG) || value < 1) {
            st = SIC_ERR_INVALID;  // unknown or malformed entry: the rest still loads
            continue;
        }
        tune_put(h, op, a, b, value, (float)ms);
    }
    fclose(f);
    return st;
}
