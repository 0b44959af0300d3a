// Reads from FASTQ on the host.  The paper's aligner takes sequencer reads
// (Section 3: paired-end lanes of 100 and 150 bases); this file parses one
// FASTQ file, or two files of mates, into batches in the packed layout the
// search takes, keeps names and qualities for SAM, and gives every base other
// than A/C/G/T a stand-in base while recording its offset.  After the search,
// mica_read_batch_filter_n recounts the hits of reads with such bases so that
// they cost one substitution wherever they fall.  No CUDA call is made here.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "read_batch_internal.h"
#include "reference_internal.h"

namespace mica {
namespace {

constexpr size_t MAX_QNAME = 254;   // SAM's QNAME limit

// Lines of a file through a 1 MiB buffer.
class LineReader {
public:
    explicit LineReader(FILE *f) : f_(f), buf_(1 << 20) {}
    ~LineReader() { fclose(f_); }
    LineReader(const LineReader &) = delete;
    LineReader &operator=(const LineReader &) = delete;

    // The next line without its end ('\n' and a '\r' before it); false at
    // the end of the file (error() tells a read error from the end).
    bool next(std::string &line)
    {
        line.clear();
        bool any = false;
        for (;;) {
            if (pos_ == end_) {
                if (eof_) return any ? finish(line) : false;
                end_ = fread(buf_.data(), 1, buf_.size(), f_);
                pos_ = 0;
                if (end_ == 0) {
                    eof_ = true;
                    error_ = ferror(f_) != 0;
                    continue;
                }
            }
            any = true;
            const char *s = buf_.data() + pos_;
            const char *nl = (const char *)memchr(s, '\n', end_ - pos_);
            if (nl) {
                line.append(s, (size_t)(nl - s));
                pos_ += (size_t)(nl - s) + 1;
                return finish(line);
            }
            line.append(s, end_ - pos_);
            pos_ = end_;
        }
    }

    bool error() const { return error_; }

private:
    static bool finish(std::string &line)
    {
        if (!line.empty() && line.back() == '\r') line.pop_back();
        return true;
    }

    FILE *f_;
    std::vector<char> buf_;
    size_t pos_ = 0, end_ = 0;
    bool eof_ = false, error_ = false;
};

struct Record {
    std::string name, seq, qual;
};

// The next record; *got = false at the end of the file.  MICA_EIO when the
// record is malformed.
int read_record(LineReader &in, Record &rec, std::string &line, bool *got)
{
    *got = false;
    do {
        if (!in.next(line)) return in.error() ? MICA_EIO : 0;
    } while (line.empty());
    if (line[0] != '@') return MICA_EIO;
    size_t e = 1;
    while (e < line.size() && line[e] != ' ' && line[e] != '\t') e++;
    rec.name.assign(line, 1, e - 1);
    if (rec.name.empty() || rec.name.size() > MAX_QNAME) return MICA_EIO;
    for (char c : rec.name)   // QNAME: [!-?A-~]
        if ((unsigned char)c < 33 || (unsigned char)c > 126 || c == '@') return MICA_EIO;
    if (!in.next(rec.seq)) return MICA_EIO;
    if (!in.next(line) || line.empty() || line[0] != '+') return MICA_EIO;
    if (!in.next(rec.qual) || rec.qual.size() != rec.seq.size()) return MICA_EIO;
    for (char c : rec.qual)
        if ((unsigned char)c < 33 || (unsigned char)c > 126) return MICA_EIO;
    *got = true;
    return 0;
}

// A mate's name without a trailing "/1" or "/2".
std::string mate_name(const std::string &name)
{
    const size_t n = name.size();
    if (n > 2 && name[n - 2] == '/' && (name[n - 1] == '1' || name[n - 1] == '2')) return name.substr(0, n - 2);
    return name;
}

int add_read(mica_read_batch &b, const Record &rec, const std::string &name, uint64_t read_no, uint8_t k)
{
    const size_t m = rec.seq.size();
    if (m == 0 || m > MICA_MAX_READ_LEN) return MICA_EINVAL;
    const size_t w0 = b.words.size(), a0 = b.amb.size();
    b.words.resize(w0 + (m + 15) / 16, 0);
    for (size_t j = 0; j < m; j++) {
        const uint8_t c = (uint8_t)rec.seq[j];
        int code = base_code(c);
        if (code < 0) {
            if (!is_letter(c) && c != '.') return MICA_EIO;
            code = (int)(splitmix64((read_no << 8) + j) >> 62);
            b.amb.push_back((uint16_t)j);
        }
        b.words[w0 + j / 16] |= (uint32_t)code << (2 * (j % 16));
    }
    if (b.amb.size() > a0) b.n_ambiguous_reads++;
    b.word_off.push_back(b.words.size());
    b.len.push_back((uint16_t)m);
    b.k.push_back(k);
    b.names.append(name);
    b.names.push_back('\0');
    b.name_off.push_back(b.names.size());
    b.quals.append(rec.qual);
    b.qual_off.push_back(b.quals.size());
    b.amb_off.push_back(b.amb.size());
    return 0;
}

}  // namespace
}  // namespace mica

struct mica_fastq {
    std::unique_ptr<mica::LineReader> in[2];
    bool paired = false;
    uint64_t next_read = 0;   // number of the next read of the file(s)
    mica::Record rec[2];
    std::string line;
};

using namespace mica;

extern "C" {

int mica_fastq_open(const char *path1, const char *path2, mica_fastq **out)
{
    if (!out) return MICA_EINVAL;
    *out = nullptr;
    if (!path1) return MICA_EINVAL;
    try {
        std::unique_ptr<mica_fastq> fq(new mica_fastq());
        for (int i = 0; i < (path2 ? 2 : 1); i++) {
            FILE *f = fopen(i ? path2 : path1, "rb");
            if (!f) return MICA_EIO;
            fq->in[i].reset(new LineReader(f));
        }
        fq->paired = path2 != nullptr;
        *out = fq.release();
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

int mica_fastq_read(mica_fastq *fq, uint64_t max_reads, uint8_t k, mica_read_batch **out)
{
    if (!out) return MICA_EINVAL;
    *out = nullptr;
    if (!fq || k > MICA_MAX_K) return MICA_EINVAL;
    if (fq->paired) max_reads &= ~1ull;
    if (max_reads < (fq->paired ? 2u : 1u)) return MICA_EINVAL;
    try {
        std::unique_ptr<mica_read_batch> b(new mica_read_batch());
        b->paired = fq->paired;
        b->word_off.push_back(0);
        b->name_off.push_back(0);
        b->qual_off.push_back(0);
        b->amb_off.push_back(0);
        Record &r1 = fq->rec[0], &r2 = fq->rec[1];
        while (b->n() < max_reads) {
            bool g1 = false, g2 = false;
            if (int rc = read_record(*fq->in[0], r1, fq->line, &g1)) return rc;
            if (!fq->paired) {
                if (!g1) break;
                if (int rc = add_read(*b, r1, r1.name, fq->next_read, k)) return rc;
                fq->next_read++;
                continue;
            }
            if (int rc = read_record(*fq->in[1], r2, fq->line, &g2)) return rc;
            if (g1 != g2) return MICA_EIO;   // files of mates of different lengths
            if (!g1) break;
            const std::string name = mate_name(r1.name);
            if (name != mate_name(r2.name)) return MICA_EIO;
            if (int rc = add_read(*b, r1, name, fq->next_read, k)) return rc;
            if (int rc = add_read(*b, r2, name, fq->next_read + 1, k)) return rc;
            fq->next_read += 2;
        }
        *out = b.release();
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

void mica_fastq_close(mica_fastq *fq) { delete fq; }

int mica_read_batch_get_view(const mica_read_batch *b, mica_read_batch_view *v)
{
    if (!b || !v) return MICA_EINVAL;
    v->n_reads = b->n();
    v->packed_reads = b->words.data();
    v->word_offsets = b->word_off.data();
    v->lengths = b->len.data();
    v->k = b->k.data();
    v->n_ambiguous_reads = b->n_ambiguous_reads;
    v->paired = b->paired ? 1u : 0u;
    return 0;
}

int mica_read_batch_read(const mica_read_batch *b, uint64_t i, const char **name, const char **qualities,
                         const uint16_t **ambiguous, uint32_t *n_ambiguous)
{
    if (!b || i >= b->n()) return MICA_EINVAL;
    if (name) *name = b->names.c_str() + b->name_off[i];
    if (qualities) *qualities = b->quals.data() + b->qual_off[i];
    if (ambiguous) *ambiguous = b->amb.data() + b->amb_off[i];
    if (n_ambiguous) *n_ambiguous = (uint32_t)(b->amb_off[i + 1] - b->amb_off[i]);
    return 0;
}

void mica_read_batch_free(mica_read_batch *b) { delete b; }

int mica_read_batch_filter_n(const mica_read_batch *b, const mica_reference *ref, uint64_t *total,
                             uint64_t *offsets, mica_hit *hits, uint64_t *n_dropped)
{
    if (n_dropped) *n_dropped = 0;
    if (!b || !ref) return MICA_EINVAL;
    const uint64_t n = b->n();
    if (n == 0) return 0;
    if (!total || !offsets) return MICA_EINVAL;
    for (uint64_t i = 0; i < n; i++)
        if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] > total[i]) return MICA_EINVAL;
    if (offsets[n] > offsets[0] && !hits) return MICA_EINVAL;
    const uint64_t text_len = ref->text.size();
    try {
        // d' of every hit of a read with ambiguous bases (0xff: unchanged),
        // decided before anything changes
        const uint64_t base0 = offsets[0];
        std::vector<uint8_t> dn(offsets[n] - base0, 0xffu);
        uint8_t codes[MICA_MAX_READ_LEN], amb[MICA_MAX_READ_LEN];
        for (uint64_t i = 0; i < n; i++) {
            if (b->amb_off[i + 1] == b->amb_off[i] || offsets[i + 1] == offsets[i]) continue;
            const uint32_t m = b->len[i];
            const uint32_t *w = b->words.data() + b->word_off[i];
            for (uint32_t j = 0; j < m; j++) {
                codes[j] = (uint8_t)((w[j >> 4] >> (2 * (j & 15))) & 3);
                amb[j] = 0;
            }
            for (uint64_t a = b->amb_off[i]; a < b->amb_off[i + 1]; a++) amb[b->amb[a]] = 1;
            for (uint64_t h = offsets[i]; h < offsets[i + 1]; h++) {
                const mica_hit &x = hits[h];
                if (x.strand > 1 || x.pos >= text_len || m > text_len - x.pos) return MICA_EINVAL;
                uint32_t raw = 0, dprime = 0;
                for (uint32_t j = 0; j < m; j++) {
                    const uint32_t ri = x.strand ? m - 1 - j : j;   // read offset at window offset j
                    const uint8_t base = x.strand ? (uint8_t)(3 - codes[ri]) : codes[ri];
                    const bool mism = ref->text[x.pos + j] != (uint8_t)"ACGT"[base];
                    raw += mism;
                    dprime += mism || amb[ri];
                }
                if (x.mm != raw && x.mm != dprime) return MICA_EINVAL;
                dn[h - base0] = (uint8_t)std::min<uint32_t>(dprime, 0xfeu);
            }
        }
        uint64_t wpos = base0, dropped = 0;
        for (uint64_t i = 0; i < n; i++) {
            const uint64_t s = offsets[i], e = offsets[i + 1];   // offsets[i + 1] not yet rewritten
            offsets[i] = wpos;
            uint64_t gone = 0;
            for (uint64_t h = s; h < e; h++) {
                const uint8_t d = dn[h - base0];
                if (d != 0xffu && d > b->k[i]) {
                    gone++;
                    continue;
                }
                mica_hit x = hits[h];
                if (d != 0xffu) x.mm = d;
                hits[wpos++] = x;   // wpos <= h
            }
            total[i] -= gone;
            dropped += gone;
        }
        offsets[n] = wpos;
        if (n_dropped) *n_dropped = dropped;
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

}  // extern "C"
