// Autotuner for the search launch: times the bidirectional kernel's compiled
// shapes and node budgets, the persistent kernel's shapes and the plain
// kernel's block size per read-length class on a sample batch and keeps the
// fastest in the index's tuning.  Tuning never changes
// results, only speed.  A small text cache keyed by (GPU name, genome length,
// length classes present, largest k) lets a later process skip the timing.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mica_internal.cuh"

namespace mica {
namespace {

uint32_t len_class_host(uint32_t m) { return m <= 64 ? 0u : m <= 128 ? 1u : m <= 192 ? 2u : 3u; }

struct DeviceBatch {
    DevBuf words, off, len, k;
    ReadsView view{};
    int upload(const uint32_t *w, const uint64_t *o, const uint16_t *l, const uint8_t *kk, uint64_t n)
    {
        uint64_t nw = o[n];
        int rc;
        if ((rc = dev_reserve(words, std::max<uint64_t>(nw, 1) * 4)) || (rc = dev_reserve(off, (n + 1) * 8)) ||
            (rc = dev_reserve(len, std::max<uint64_t>(n, 1) * 2)) || (rc = dev_reserve(k, std::max<uint64_t>(n, 1))))
            return rc;
        if (nw) MICA_CUDA_TRY(cudaMemcpy(words.p, w, nw * 4, cudaMemcpyHostToDevice));
        MICA_CUDA_TRY(cudaMemcpy(off.p, o, (n + 1) * 8, cudaMemcpyHostToDevice));
        if (n) {
            MICA_CUDA_TRY(cudaMemcpy(len.p, l, n * 2, cudaMemcpyHostToDevice));
            MICA_CUDA_TRY(cudaMemcpy(k.p, kk, n, cudaMemcpyHostToDevice));
        }
        view = ReadsView{(const uint32_t *)words.p, (const uint64_t *)off.p, (const uint16_t *)len.p,
                         (const uint8_t *)k.p, n};
        return 0;
    }
    ~DeviceBatch() { dev_release(words); dev_release(off); dev_release(len); dev_release(k); }
};

// best (minimum) search-kernel time of `repeats` runs after one warm-up
int time_search(mica_index *idx, Workspace &ws, const ReadsView &rd, int kernel, uint32_t hit_cap,
                uint32_t repeats, float *best)
{
    mica_align_params p;
    mica_align_params_default(&p);
    p.kernel = kernel;
    p.hit_cap = hit_cap;
    *best = 1e30f;
    for (uint32_t r = 0; r <= repeats; r++) {
        mica_stats st{};
        uint64_t nh = 0;
        if (int rc = align_on_device(idx, ws, st, rd, p, 0, &nh, false)) return rc;
        if (r > 0) *best = std::min(*best, st.kernel_ms);
    }
    return 0;
}

std::string cache_key(const mica_index *idx, uint32_t classes, uint32_t kmax)
{
    cudaDeviceProp prop;
    char name[256] = "unknown";
    if (cudaGetDeviceProperties(&prop, idx->device) == cudaSuccess) snprintf(name, sizeof(name), "%s", prop.name);
    for (char *c = name; *c; c++)
        if (*c == '\t' || *c == '\n') *c = ' ';
    char key[400];
    snprintf(key, sizeof(key), "%s\t%llu\t%u\t%u\t%u", name, (unsigned long long)idx->n, idx->params.kmer_q, classes,
             kmax);
    return key;
}

}  // namespace
}  // namespace mica

using namespace mica;

extern "C" {

int mica_autotune(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                  const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint32_t hit_cap, uint32_t repeats,
                  mica_tuning *out)
{
    if (!idx || !word_offsets || n_reads == 0 || !packed_reads || !lengths || !k) return MICA_EINVAL;
    if (int rc = validate_host_batch(idx, word_offsets, lengths, k, n_reads)) return rc;
    if (repeats == 0) repeats = 1;
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    mica_tuning best = idx->tuning;
    Workspace ws;
    int rc = 0;
    {
        DeviceBatch all;
        if ((rc = all.upload(packed_reads, word_offsets, lengths, k, n_reads))) goto done;
        float tbest = 1e30f;
        // bidirectional shapes (task slots and warps per CTA) and node budgets
        if (bidir_available(idx)) {
            const uint32_t budgets[] = {1024, 4096};
            for (int s = 0; s < bidir_shape_count(); s++)
                for (uint32_t b : budgets) {
                    idx->tuning.bidir_shape = s;
                    idx->tuning.bidir_budget = b;
                    float t;
                    if ((rc = time_search(idx, ws, all.view, MICA_KERNEL_BIDIRECTIONAL, hit_cap, repeats, &t)))
                        goto done;
                    if (t < tbest) { tbest = t; best.bidir_shape = s; best.bidir_budget = b; }
                }
            idx->tuning.bidir_shape = best.bidir_shape;
            idx->tuning.bidir_budget = best.bidir_budget;
        }
        // persistent shapes
        tbest = 1e30f;
        for (int s = 0; s < search_shape_count(); s++) {
            idx->tuning.shape = s;
            float t;
            if ((rc = time_search(idx, ws, all.view, MICA_KERNEL_PERSISTENT, hit_cap, repeats, &t))) goto done;
            if (t < tbest) { tbest = t; best.shape = s; }
        }
        idx->tuning.shape = best.shape;
        // plain block size over the whole batch
        const uint32_t blocks[] = {64, 128, 256, 512};
        tbest = 1e30f;
        for (uint32_t b : blocks) {
            idx->tuning.plain_block = b;
            float t;
            if ((rc = time_search(idx, ws, all.view, MICA_KERNEL_PLAIN, hit_cap, repeats, &t))) goto done;
            if (t < tbest) { tbest = t; best.plain_block = b; }
        }
        idx->tuning.plain_block = best.plain_block;
    }
    // plain block size per read-length class, on that class's reads alone
    for (uint32_t c = 0; c < LEN_CLASSES; c++) {
        std::vector<uint32_t> w;
        std::vector<uint64_t> o(1, 0);
        std::vector<uint16_t> l;
        std::vector<uint8_t> kk;
        for (uint64_t i = 0; i < n_reads; i++) {
            if (len_class_host(lengths[i]) != c) continue;
            uint32_t nw = (lengths[i] + 15) / 16;
            w.insert(w.end(), packed_reads + word_offsets[i], packed_reads + word_offsets[i] + nw);
            o.push_back(w.size());
            l.push_back(lengths[i]);
            kk.push_back(k[i]);
        }
        best.plain_block_len[c] = 0;
        if (l.empty()) continue;
        DeviceBatch sub;
        if ((rc = sub.upload(w.data(), o.data(), l.data(), kk.data(), l.size()))) goto done;
        float tbest = 1e30f;
        for (uint32_t b : {64u, 128u, 256u, 512u}) {
            idx->tuning.plain_block = b;
            float t;
            if ((rc = time_search(idx, ws, sub.view, MICA_KERNEL_PLAIN, hit_cap, repeats, &t))) goto done;
            if (t < tbest) { tbest = t; best.plain_block_len[c] = b; }
        }
    }
done:
    free_workspace(ws);
    if (rc) {
        idx->tuning = best;   // keep what was decided so far
        return rc;
    }
    idx->tuning = best;
    if (out) *out = best;
    return 0;
}

int mica_tuning_cache_store(const char *path, const mica_index *idx, uint32_t length_classes, uint32_t kmax,
                            const mica_tuning *t)
{
    if (!path || !idx || !t) return MICA_EINVAL;
    std::string key = cache_key(idx, length_classes, kmax);
    // keep other keys, replace this one
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[1024];
        while (fgets(line, sizeof(line), f)) {
            std::string s(line);
            if (s.compare(0, key.size() + 1, key + "\t") != 0) keep.push_back(s);
        }
        fclose(f);
    }
    FILE *f = fopen(path, "w");
    if (!f) return MICA_EIO;
    for (auto &s : keep) fputs(s.c_str(), f);
    fprintf(f, "%s\t%d %u %u %u %u %u %u %d %u %u %d\n", key.c_str(), t->shape, t->plain_block, t->plain_budget,
            t->plain_block_len[0], t->plain_block_len[1], t->plain_block_len[2], t->plain_block_len[3], t->prefetch,
            t->bidir_budget, t->bidir_verify, t->bidir_shape);
    return fclose(f) == 0 ? 0 : MICA_EIO;
}

int mica_tuning_cache_lookup(const char *path, const mica_index *idx, uint32_t length_classes, uint32_t kmax,
                             mica_tuning *t)
{
    if (!path || !idx || !t) return MICA_EINVAL;
    std::string key = cache_key(idx, length_classes, kmax) + "\t";
    FILE *f = fopen(path, "r");
    if (!f) return MICA_ENOTFOUND;
    char line[1024];
    int rc = MICA_ENOTFOUND;
    while (fgets(line, sizeof(line), f)) {
        if (strncmp(line, key.c_str(), key.size()) != 0) continue;
        mica_tuning x{};
        // lines written before the bidirectional fields were added hold eight or nine numbers
        x.bidir_budget = 0;
        x.bidir_verify = 0;
        x.bidir_shape = -1;
        if (sscanf(line + key.size(), "%d %u %u %u %u %u %u %d %u %u %d", &x.shape, &x.plain_block, &x.plain_budget,
                   &x.plain_block_len[0], &x.plain_block_len[1], &x.plain_block_len[2], &x.plain_block_len[3],
                   &x.prefetch, &x.bidir_budget, &x.bidir_verify, &x.bidir_shape) >= 8 &&
            x.shape >= -1 && x.shape < search_shape_count() && x.prefetch >= -1 && x.prefetch <= 1 &&
            x.bidir_shape >= -1 && x.bidir_shape < bidir_shape_count()) {
            *t = x;
            rc = 0;
        }
    }
    fclose(f);
    return rc;
}

}  // extern "C"
