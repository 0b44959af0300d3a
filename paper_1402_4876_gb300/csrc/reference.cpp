// Reference sequences on the host.  The paper's aligner places reads on a
// reference genome (Section 2); a real reference comes as named contigs whose
// bytes may hold N and other IUPAC codes, while the index searches one text
// over {A,C,G,T}.  This file concatenates the contigs into that text G,
// replaces each ambiguous byte by a base derived from its coordinate,
// records the ambiguous runs, decides which windows of G are placements on
// the reference, filters hit lists by that rule and keeps a binary copy.
// No CUDA call is made here.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <unordered_set>

#include "host_parallel.h"
#include "reference_internal.h"

namespace mica {
namespace {

constexpr uint64_t MAX_TEXT = (1ull << 32) - 2;   // the index keeps |G| + 1 < 2^32 rows
constexpr uint64_t MAX_NAME = 1u << 16;
constexpr char FILE_MAGIC[8] = {'M', 'I', 'C', 'A', 'R', 'E', 'F', '1'};

inline uint8_t replacement_base(uint64_t coord) { return "ACGT"[splitmix64(coord) >> 62]; }

inline bool is_space(uint8_t c) { return c == ' ' || c == '\t' || c == '\r' || c == '\n' || c == '\v' || c == '\f'; }

// Append one sequence byte to G (the caller checks the length limit).
inline void push_base(mica_reference &r, uint8_t c)
{
    const uint64_t j = r.text.size();
    if (base_code(c) >= 0) {
        r.text.push_back((uint8_t)(c & ~0x20));   // upper case
        return;
    }
    if (!r.amb_end.empty() && r.amb_end.back() == j) {
        r.amb_end.back() = j + 1;
    } else {
        r.amb_start.push_back(j);
        r.amb_end.push_back(j + 1);
    }
    r.text.push_back(replacement_base(j));
}

// Checks shared by every way of making a reference.
int check_contigs(const mica_reference &r)
{
    const uint64_t nc = r.names.size();
    if (nc == 0 || nc >= (1ull << 31) || r.start.size() != nc + 1 || r.start[0] != 0 ||
        r.start[nc] != r.text.size() || r.text.size() > MAX_TEXT)
        return MICA_EINVAL;
    std::unordered_set<std::string> seen;
    seen.reserve(nc);
    for (uint64_t i = 0; i < nc; i++) {
        if (r.start[i + 1] <= r.start[i] || !sam_name_ok(r.names[i]) || !seen.insert(r.names[i]).second)
            return MICA_EINVAL;
    }
    return 0;
}

struct FileCloser {
    void operator()(FILE *f) const { if (f) fclose(f); }
};
using File = std::unique_ptr<FILE, FileCloser>;

template <typename T> bool put(FILE *f, const T &v) { return fwrite(&v, sizeof(T), 1, f) == 1; }
template <typename T> bool get(FILE *f, T &v) { return fread(&v, sizeof(T), 1, f) == 1; }

int read_fasta(FILE *f, mica_reference &r)
{
    enum { START, NAME, HEADER_REST, COMMENT, SEQ } state = START;
    bool line_start = true, in_record = false;
    std::string name;
    std::vector<uint8_t> buf(1 << 20);
    auto end_record = [&]() -> int {
        if (!in_record) return 0;
        if (r.text.size() == r.start.back()) return MICA_EIO;   // empty record
        r.start.push_back(r.text.size());
        return 0;
    };
    for (;;) {
        const size_t got = fread(buf.data(), 1, buf.size(), f);
        if (got == 0) break;
        for (size_t t = 0; t < got; t++) {
            const uint8_t c = buf[t];
            if (line_start && c == '>') {
                if (int rc = end_record()) return rc;
                name.clear();
                state = NAME;
                line_start = false;
                continue;
            }
            if (line_start && c == ';') {
                state = COMMENT;
                line_start = false;
                continue;
            }
            switch (state) {
            case NAME:
                if (is_space(c)) {
                    if (name.empty() || !sam_name_ok(name)) return MICA_EIO;
                    r.names.push_back(name);
                    in_record = true;
                    state = c == '\n' ? SEQ : HEADER_REST;
                } else {
                    if (name.size() >= MAX_NAME) return MICA_EIO;
                    name.push_back((char)c);
                }
                break;
            case HEADER_REST:
                if (c == '\n') state = SEQ;
                break;
            case COMMENT:
                if (c == '\n') state = in_record ? SEQ : START;
                break;
            case START:
                if (!is_space(c)) return MICA_EIO;   // bytes before the first record
                break;
            case SEQ:
                if (is_letter(c)) {
                    if (r.text.size() >= MAX_TEXT) return MICA_EINVAL;
                    push_base(r, c);
                } else if (!is_space(c)) {
                    return MICA_EIO;
                }
                break;
            }
            line_start = c == '\n';
        }
    }
    if (ferror(f)) return MICA_EIO;
    if (state == NAME) {   // a header line at the very end of the file
        if (name.empty() || !sam_name_ok(name)) return MICA_EIO;
        r.names.push_back(name);
        in_record = true;
    }
    if (int rc = end_record()) return rc;
    if (r.names.empty()) return MICA_EIO;
    return check_contigs(r) ? MICA_EIO : 0;
}

}  // namespace

bool sam_name_ok(const std::string &s)
{
    if (s.empty()) return false;
    for (size_t i = 0; i < s.size(); i++) {
        const unsigned char c = (unsigned char)s[i];
        if (c < 33 || c > 126 || strchr("\"'(),<>[\\]`{}", c)) return false;
        if (i == 0 && (c == '*' || c == '=')) return false;
    }
    return true;
}

int32_t reference_place(const mica_reference &r, uint64_t pos, uint64_t span)
{
    const uint64_t n = r.text.size();
    if (span == 0 || pos >= n || span > n - pos) return PLACE_OUT_OF_RANGE;
    // the contig holding pos: the last start <= pos (start[0] = 0)
    const size_t c = (size_t)(std::upper_bound(r.start.begin(), r.start.end() - 1, pos) - r.start.begin()) - 1;
    if (pos + span > r.start[c + 1]) return PLACE_OFF_REFERENCE;
    // the first ambiguous run ending after pos must start at or after the window's end
    const size_t j = (size_t)(std::upper_bound(r.amb_end.begin(), r.amb_end.end(), pos) - r.amb_end.begin());
    if (j < r.amb_end.size() && r.amb_start[j] < pos + span) return PLACE_OFF_REFERENCE;
    return (int32_t)c;
}

}  // namespace mica

using namespace mica;

extern "C" {

int mica_reference_create(const uint8_t *sequence, uint64_t len, const uint64_t *contig_lengths,
                          const char *const *names, uint64_t n_contigs, mica_reference **out)
{
    if (!out) return MICA_EINVAL;
    *out = nullptr;
    if (n_contigs == 0 || !contig_lengths || (len && !sequence) || len > MAX_TEXT) return MICA_EINVAL;
    try {
        std::unique_ptr<mica_reference> r(new mica_reference());
        r->start.push_back(0);
        uint64_t sum = 0;
        for (uint64_t i = 0; i < n_contigs; i++) {
            if (contig_lengths[i] == 0 || contig_lengths[i] > len - sum) return MICA_EINVAL;
            sum += contig_lengths[i];
            r->start.push_back(sum);
            if (names) {
                if (!names[i]) return MICA_EINVAL;
                r->names.emplace_back(names[i]);
            } else {
                r->names.push_back("contig" + std::to_string(i + 1));
            }
        }
        if (sum != len) return MICA_EINVAL;
        r->text.reserve(len);
        for (uint64_t j = 0; j < len; j++) push_base(*r, sequence[j]);
        if (int rc = check_contigs(*r)) return rc;
        *out = r.release();
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

int mica_reference_read_fasta(const char *path, mica_reference **out)
{
    if (!out || !path) return MICA_EINVAL;
    *out = nullptr;
    File f(fopen(path, "rb"));
    if (!f) return MICA_EIO;
    try {
        std::unique_ptr<mica_reference> r(new mica_reference());
        r->start.push_back(0);
        if (fseek(f.get(), 0, SEEK_END) == 0) {
            const long size = ftell(f.get());
            if (size > 0) r->text.reserve(std::min<uint64_t>((uint64_t)size, MAX_TEXT));
            rewind(f.get());
        }
        if (int rc = read_fasta(f.get(), *r)) return rc;
        *out = r.release();
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

int mica_reference_save(const mica_reference *ref, const char *path)
{
    if (!ref || !path) return MICA_EINVAL;
    File f(fopen(path, "wb"));
    if (!f) return MICA_EIO;
    FILE *F = f.get();
    const uint64_t nc = ref->names.size(), n = ref->text.size(), nr = ref->amb_start.size();
    bool ok = fwrite(FILE_MAGIC, 1, 8, F) == 8 && put(F, nc) && put(F, n) && put(F, nr);
    for (uint64_t i = 0; ok && i < nc; i++) {
        const uint64_t nl = ref->names[i].size(), cl = ref->start[i + 1] - ref->start[i];
        ok = put(F, nl) && fwrite(ref->names[i].data(), 1, nl, F) == nl && put(F, cl);
    }
    for (uint64_t j = 0; ok && j < nr; j++) ok = put(F, ref->amb_start[j]) && put(F, ref->amb_end[j]);
    // G at 2 bits per base, base j in bits 2 (j mod 4) of byte j / 4
    std::vector<uint8_t> packed;
    for (uint64_t b = 0; ok && b < n; b += 1u << 22) {
        const uint64_t e = std::min<uint64_t>(n, b + (1u << 22));
        packed.assign((e - b + 3) / 4, 0);
        for (uint64_t j = b; j < e; j++)
            packed[(j - b) >> 2] |= (uint8_t)(base_code(ref->text[j]) << (2 * ((j - b) & 3)));
        ok = fwrite(packed.data(), 1, packed.size(), F) == packed.size();
    }
    if (!ok) return MICA_EIO;
    return fclose(f.release()) == 0 ? 0 : MICA_EIO;
}

int mica_reference_load(const char *path, mica_reference **out)
{
    if (!out || !path) return MICA_EINVAL;
    *out = nullptr;
    File f(fopen(path, "rb"));
    if (!f) return MICA_EIO;
    FILE *F = f.get();
    try {
        char magic[8];
        uint64_t nc = 0, n = 0, nr = 0;
        if (fread(magic, 1, 8, F) != 8 || memcmp(magic, FILE_MAGIC, 8) != 0 || !get(F, nc) || !get(F, n) ||
            !get(F, nr) || n > MAX_TEXT || nc == 0 || nc > n || nr > n)
            return MICA_EIO;
        std::unique_ptr<mica_reference> r(new mica_reference());
        r->start.push_back(0);
        for (uint64_t i = 0; i < nc; i++) {
            uint64_t nl = 0, cl = 0;
            if (!get(F, nl) || nl == 0 || nl > MAX_NAME) return MICA_EIO;
            std::string name(nl, '\0');
            if (fread(&name[0], 1, nl, F) != nl || !get(F, cl) || cl == 0 || cl > n - r->start.back())
                return MICA_EIO;
            r->names.push_back(std::move(name));
            r->start.push_back(r->start.back() + cl);
        }
        if (r->start.back() != n) return MICA_EIO;
        uint64_t prev_end = 0;
        for (uint64_t j = 0; j < nr; j++) {
            uint64_t s = 0, e = 0;
            if (!get(F, s) || !get(F, e) || s >= e || e > n || (j && s <= prev_end)) return MICA_EIO;
            r->amb_start.push_back(s);
            r->amb_end.push_back(e);
            prev_end = e;
        }
        r->text.resize(n);
        std::vector<uint8_t> packed;
        for (uint64_t b = 0; b < n; b += 1u << 22) {
            const uint64_t e = std::min<uint64_t>(n, b + (1u << 22));
            packed.resize((e - b + 3) / 4);
            if (fread(packed.data(), 1, packed.size(), F) != packed.size()) return MICA_EIO;
            for (uint64_t j = b; j < e; j++)
                r->text[j] = (uint8_t)"ACGT"[(packed[(j - b) >> 2] >> (2 * ((j - b) & 3))) & 3];
        }
        if (fgetc(F) != EOF) return MICA_EIO;   // trailing bytes
        for (uint64_t j = 0; j < nr; j++)       // replaced bases are the coordinate's own
            for (uint64_t x = r->amb_start[j]; x < r->amb_end[j]; x++)
                if (r->text[x] != replacement_base(x)) return MICA_EIO;
        if (check_contigs(*r)) return MICA_EIO;
        *out = r.release();
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

void mica_reference_free(mica_reference *ref) { delete ref; }

int mica_reference_get_info(const mica_reference *ref, mica_reference_info *info)
{
    if (!ref || !info) return MICA_EINVAL;
    info->length = ref->text.size();
    info->n_contigs = ref->names.size();
    info->n_ambiguous_runs = ref->amb_start.size();
    uint64_t nb = 0;
    for (size_t j = 0; j < ref->amb_start.size(); j++) nb += ref->amb_end[j] - ref->amb_start[j];
    info->ambiguous_bases = nb;
    return 0;
}

int mica_reference_text(const mica_reference *ref, const uint8_t **acgt, uint64_t *len)
{
    if (!ref || !acgt || !len) return MICA_EINVAL;
    *acgt = ref->text.data();
    *len = ref->text.size();
    return 0;
}

int mica_reference_contig(const mica_reference *ref, uint64_t i, const char **name, uint64_t *start,
                          uint64_t *length)
{
    if (!ref || i >= ref->names.size()) return MICA_EINVAL;
    if (name) *name = ref->names[i].c_str();
    if (start) *start = ref->start[i];
    if (length) *length = ref->start[i + 1] - ref->start[i];
    return 0;
}

int mica_reference_ambiguous_run(const mica_reference *ref, uint64_t j, uint64_t *start, uint64_t *length)
{
    if (!ref || j >= ref->amb_start.size()) return MICA_EINVAL;
    if (start) *start = ref->amb_start[j];
    if (length) *length = ref->amb_end[j] - ref->amb_start[j];
    return 0;
}

int mica_reference_locate(const mica_reference *ref, const uint32_t *pos, const uint16_t *span, uint64_t n,
                          int32_t *contig, uint32_t *local)
{
    if (!ref || (n && (!pos || !span || !contig || !local))) return MICA_EINVAL;
    for (uint64_t i = 0; i < n; i++)
        if (reference_place(*ref, pos[i], span[i]) == PLACE_OUT_OF_RANGE) return MICA_EINVAL;
    for (uint64_t i = 0; i < n; i++) {
        const int32_t c = reference_place(*ref, pos[i], span[i]);
        contig[i] = c;
        local[i] = c >= 0 ? (uint32_t)(pos[i] - ref->start[c]) : 0;
    }
    return 0;
}

int mica_reference_filter(const mica_reference *ref, const uint16_t *lengths, uint64_t n_reads, uint64_t *total,
                          uint64_t *offsets, mica_hit *hits, uint64_t *n_dropped)
{
    if (n_dropped) *n_dropped = 0;
    if (!ref || (n_reads && (!lengths || !total || !offsets))) return MICA_EINVAL;
    if (n_reads == 0) return 0;
    for (uint64_t i = 0; i < n_reads; i++)
        if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] > total[i]) return MICA_EINVAL;
    if (offsets[n_reads] > offsets[0] && !hits) return MICA_EINVAL;
    try {
        // decide every hit first (reads in chunks on host threads), so that
        // bad input changes nothing
        const uint64_t base0 = offsets[0];
        std::vector<uint8_t> keep(offsets[n_reads] - base0);
        const uint64_t chunk = 16384, n_chunks = (n_reads + chunk - 1) / chunk;
        std::atomic<bool> bad{false};
        parallel_chunks(n_chunks, host_threads(), [&](uint64_t c) {
            for (uint64_t i = c * chunk; i < std::min(n_reads, (c + 1) * chunk); i++)
                for (uint64_t h = offsets[i]; h < offsets[i + 1]; h++) {
                    const int32_t pl = reference_place(*ref, hits[h].pos, lengths[i]);
                    if (pl == PLACE_OUT_OF_RANGE) bad = true;
                    keep[h - base0] = pl >= 0;
                }
        });
        if (bad) return MICA_EINVAL;
        uint64_t w = base0, dropped = 0;
        for (uint64_t i = 0; i < n_reads; i++) {
            const uint64_t b = offsets[i], e = offsets[i + 1];   // offsets[i + 1] not yet rewritten
            offsets[i] = w;
            uint64_t gone = 0;
            for (uint64_t h = b; h < e; h++) {
                if (keep[h - base0]) hits[w++] = hits[h];   // w <= h
                else gone++;
            }
            total[i] -= gone;
            dropped += gone;
        }
        offsets[n_reads] = w;
        if (n_dropped) *n_dropped = dropped;
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

}  // extern "C"
