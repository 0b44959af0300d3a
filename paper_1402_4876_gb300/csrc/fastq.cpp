// Reads from FASTQ on the host.  The paper's aligner takes sequencer reads
// (Section 3: paired-end lanes of 100 and 150 bases); this file parses one
// FASTQ file, or two files of mates, into batches in the packed layout the
// search takes, keeps names and qualities for SAM, and gives every base other
// than A/C/G/T a stand-in base while recording its offset.  After the search,
// mica_read_batch_filter_n recounts the hits of reads with such bases so that
// they cost one substitution wherever they fall.  No CUDA call is made here.
//
// A batch is read in two steps: the file is read in large blocks whose line
// ends are found on all host threads, and cut into records (one thread,
// over those offsets); then the records are checked and packed in chunks on
// all host threads and the chunks joined in file order.  After a full batch
// a background thread reads and indexes about as many bytes again, so that
// the reading overlaps whatever the caller does with the batch.
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "host_parallel.h"
#include "read_batch_internal.h"
#include "reference_internal.h"

namespace mica {
namespace {

constexpr size_t MAX_QNAME = 254;        // SAM's QNAME limit
constexpr size_t BLOCK = 64u << 20;      // bytes read at a time
constexpr uint64_t CHUNK_RECORDS = 8192; // records packed per task (even)

// One FASTQ file: bytes read but not yet consumed by a batch, and the
// offsets of their line ends, found on host threads block by block.
struct Input {
    FILE *f = nullptr;
    char *data = nullptr;       // malloc'd, grown with realloc (never zero-filled)
    size_t cap = 0, size = 0;   // capacity and valid bytes
    size_t base = 0;            // bytes before base are consumed
    std::vector<size_t> nl;     // offsets of '\n' in [0, size), ascending
    size_t li = 0;              // nl[li] ends the line the cursor is on
    bool eof = false;
    bool error = false;

    Input() = default;
    Input(const Input &) = delete;
    Input &operator=(const Input &) = delete;
    ~Input()
    {
        if (f) fclose(f);
        free(data);
    }

    // Reads up to BLOCK more bytes and indexes their line ends; false when
    // there are none.
    bool fill()
    {
        if (eof) return false;
        if (cap < size + BLOCK) {
            const size_t ncap = std::max(size + BLOCK, 2 * cap);
            char *p = (char *)realloc(data, ncap);
            if (!p) throw std::bad_alloc();
            data = p;
            cap = ncap;
        }
        const size_t got = fread(data + size, 1, BLOCK, f);
        if (got < BLOCK) {
            eof = true;
            error = ferror(f) != 0;
        }
        index(size, size + got);
        size += got;
        return got > 0;
    }

    // Appends the line ends of [a, e) to nl, segments scanned in parallel.
    void index(size_t a, size_t e)
    {
        const uint64_t segs = std::max<uint64_t>(1, std::min<uint64_t>(host_threads(), (e - a) >> 20));
        std::vector<std::vector<size_t>> found(segs);
        const size_t step = (e - a + segs - 1) / segs;
        parallel_chunks(segs, host_threads(), [&](uint64_t t) {
            try {
                const size_t s0 = a + t * step, s1 = std::min(e, s0 + step);
                for (size_t p = s0; p < s1;) {
                    const char *q = (const char *)memchr(data + p, '\n', s1 - p);
                    if (!q) break;
                    found[t].push_back((size_t)(q - data));
                    p = (size_t)(q - data) + 1;
                }
            } catch (const std::bad_alloc &) {
                found[t].assign(1, SIZE_MAX);   // reported below
            }
        });
        for (auto &v : found) {
            if (!v.empty() && v[0] == SIZE_MAX) throw std::bad_alloc();
            nl.insert(nl.end(), v.begin(), v.end());
        }
    }

    // The line starting at *pos as [*a, *b) without its end ('\n' and a '\r'
    // before it); advances *pos past it.  false at the end of the input.
    bool line(size_t *pos, size_t *a, size_t *b)
    {
        while (li == nl.size())
            if (!fill()) break;
        if (li < nl.size()) {
            *a = *pos;
            *b = nl[li++];
            *pos = *b + 1;
        } else {
            if (*pos >= size) return false;
            *a = *pos;   // a last line without '\n'
            *b = size;
            *pos = size;
        }
        if (*b > *a && data[*b - 1] == '\r') --*b;
        return true;
    }

    // Consumes the bytes before `pos` (a line start reached by the cursor);
    // they are dropped once they outnumber the rest, so each byte moves at
    // most about once.
    void consume(size_t pos)
    {
        base = pos;
        if (base <= size - base) return;
        memmove(data, data + base, size - base);
        size -= base;
        nl.erase(nl.begin(), nl.begin() + (ptrdiff_t)li);
        for (size_t &x : nl) x -= base;
        li = 0;
        base = 0;
    }
};

// A record's lines as byte ranges of its Input's data.
struct Span {
    size_t h0, h1, s0, s1, q0, q1;   // header (with '@'), bases, qualities
};

// Cuts up to `want` records from `in` starting at *pos.  MICA_EIO on a
// record without its four lines or a third line not starting with '+'.
int cut_records(Input &in, size_t *pos, uint64_t want, std::vector<Span> &out)
{
    size_t a, b;
    while (out.size() < want) {
        Span s;
        do {
            if (!in.line(pos, &a, &b)) return in.error ? MICA_EIO : 0;
        } while (a == b);   // blank lines between records
        s.h0 = a;
        s.h1 = b;
        if (!in.line(pos, &s.s0, &s.s1)) return MICA_EIO;
        if (!in.line(pos, &a, &b) || a == b || in.data[a] != '+') return MICA_EIO;
        if (!in.line(pos, &s.q0, &s.q1)) return MICA_EIO;
        out.push_back(s);
    }
    return 0;
}

// The reads of one chunk of records, joined into the batch afterwards.
struct Part {
    std::vector<uint32_t> words;
    std::vector<uint64_t> word_end;   // per read, relative to the part
    std::vector<uint16_t> len;
    std::string names;                // NUL-terminated names back to back
    std::vector<uint64_t> name_end;
    std::string quals;
    std::vector<uint16_t> amb;
    std::vector<uint64_t> amb_end;
    uint64_t n_ambiguous_reads = 0;
    int err = 0;
};

// The name of a record (first word of its header), checked as a QNAME;
// a trailing "/1" or "/2" is dropped for mates.
int record_name(const Input &in, const Span &s, bool mate, const char **p, size_t *n)
{
    if (s.h1 == s.h0 || in.data[s.h0] != '@') return MICA_EIO;
    size_t e = s.h0 + 1;
    while (e < s.h1 && in.data[e] != ' ' && in.data[e] != '\t') e++;
    const char *name = in.data + s.h0 + 1;
    size_t len = e - s.h0 - 1;
    if (len == 0 || len > MAX_QNAME) return MICA_EIO;
    for (size_t j = 0; j < len; j++) {   // QNAME: [!-?A-~]
        const unsigned char c = (unsigned char)name[j];
        if (c < 33 || c > 126 || c == '@') return MICA_EIO;
    }
    if (mate && len > 2 && name[len - 2] == '/' && (name[len - 1] == '1' || name[len - 1] == '2')) len -= 2;
    *p = name;
    *n = len;
    return 0;
}

int pack_record(Part &part, const Input &in, const Span &s, const char *name, size_t name_len, uint64_t read_no)
{
    const size_t m = s.s1 - s.s0;
    if (m == 0 || m > MICA_MAX_READ_LEN) return MICA_EINVAL;
    if (s.q1 - s.q0 != m) return MICA_EIO;
    const char *seq = in.data + s.s0, *qual = in.data + s.q0;
    for (size_t j = 0; j < m; j++)
        if ((unsigned char)qual[j] < 33 || (unsigned char)qual[j] > 126) return MICA_EIO;
    const size_t w0 = part.words.size(), a0 = part.amb.size();
    part.words.resize(w0 + (m + 15) / 16, 0);
    uint32_t *w = part.words.data() + w0;
    for (size_t j = 0; j < m; j++) {
        const uint8_t c = (uint8_t)seq[j];
        int code = base_code(c);
        if (code < 0) {
            if (!is_letter(c) && c != '.') return MICA_EIO;
            code = (int)(splitmix64((read_no << 8) + j) >> 62);
            part.amb.push_back((uint16_t)j);
        }
        w[j >> 4] |= (uint32_t)code << (2 * (j & 15));
    }
    if (part.amb.size() > a0) part.n_ambiguous_reads++;
    part.word_end.push_back(part.words.size());
    part.len.push_back((uint16_t)m);
    part.names.append(name, name_len);
    part.names.push_back('\0');
    part.name_end.push_back(part.names.size());
    part.quals.append(qual, m);
    part.amb_end.push_back(part.amb.size());
    return 0;
}

// Packs the reads of records [a, e) (pair indices when paired) into `part`.
void pack_chunk(Part &part, Input *const in[2], const std::vector<Span> *spans, bool paired, uint64_t a,
                uint64_t e, uint64_t first_read)
{
    for (uint64_t r = a; r < e && !part.err; r++) {
        if (!paired) {
            const char *name;
            size_t nl;
            part.err = record_name(*in[0], spans[0][r], false, &name, &nl);
            if (!part.err) part.err = pack_record(part, *in[0], spans[0][r], name, nl, first_read + r);
            continue;
        }
        const char *n1, *n2;
        size_t l1, l2;
        part.err = record_name(*in[0], spans[0][r], true, &n1, &l1);
        if (!part.err) part.err = record_name(*in[1], spans[1][r], true, &n2, &l2);
        if (!part.err && (l1 != l2 || memcmp(n1, n2, l1) != 0)) part.err = MICA_EIO;   // mates' names differ
        if (!part.err) part.err = pack_record(part, *in[0], spans[0][r], n1, l1, first_read + 2 * r);
        if (!part.err) part.err = pack_record(part, *in[1], spans[1][r], n1, l1, first_read + 2 * r + 1);
    }
}

// Joins the parts in order: every array is sized once, then each part is
// copied into its place on host threads.
void join_parts(mica_read_batch &b, const std::vector<Part> &parts, uint8_t k)
{
    const size_t np = parts.size();
    std::vector<uint64_t> r0(np + 1, 0), w0(np + 1, 0), n0(np + 1, 0), q0(np + 1, 0), a0(np + 1, 0);
    for (size_t c = 0; c < np; c++) {
        const Part &p = parts[c];
        r0[c + 1] = r0[c] + p.len.size();
        w0[c + 1] = w0[c] + p.words.size();
        n0[c + 1] = n0[c] + p.names.size();
        q0[c + 1] = q0[c] + p.quals.size();
        a0[c + 1] = a0[c] + p.amb.size();
        b.n_ambiguous_reads += p.n_ambiguous_reads;
    }
    const uint64_t n = r0[np];
    b.words.resize(w0[np]);
    b.names.resize(n0[np]);
    b.quals.resize(q0[np]);
    b.amb.resize(a0[np]);
    b.len.resize(n);
    b.k.assign(n, k);
    b.word_off.assign(n + 1, 0);
    b.name_off.assign(n + 1, 0);
    b.qual_off.assign(n + 1, 0);
    b.amb_off.assign(n + 1, 0);
    parallel_chunks(np, host_threads(), [&](uint64_t c) {
        const Part &p = parts[c];
        std::copy(p.words.begin(), p.words.end(), b.words.begin() + (ptrdiff_t)w0[c]);
        std::copy(p.names.begin(), p.names.end(), b.names.begin() + (ptrdiff_t)n0[c]);
        std::copy(p.quals.begin(), p.quals.end(), b.quals.begin() + (ptrdiff_t)q0[c]);
        std::copy(p.amb.begin(), p.amb.end(), b.amb.begin() + (ptrdiff_t)a0[c]);
        std::copy(p.len.begin(), p.len.end(), b.len.begin() + (ptrdiff_t)r0[c]);
        uint64_t q = q0[c];
        for (size_t i = 0; i < p.len.size(); i++) {
            const uint64_t r = r0[c] + i + 1;
            b.word_off[r] = w0[c] + p.word_end[i];
            b.name_off[r] = n0[c] + p.name_end[i];
            q += p.len[i];
            b.qual_off[r] = q;
            b.amb_off[r] = a0[c] + p.amb_end[i];
        }
    });
}

}  // namespace
}  // namespace mica

struct mica_fastq {
    mica::Input in[2];
    bool paired = false;
    uint64_t next_read = 0;   // number of the next read of the file(s)
    std::vector<mica::Span> spans[2];
    // reads and indexes the next batch's bytes while the caller works on the
    // last batch; joined before the inputs are touched again
    std::thread ahead;

    void join_ahead()
    {
        if (ahead.joinable()) ahead.join();
    }
    ~mica_fastq() { join_ahead(); }
};

namespace mica {
namespace {

// Fills each input until it holds `bytes` unconsumed bytes (or its end).
void read_ahead(mica_fastq *fq, size_t bytes)
{
    try {
        for (int i = 0; i < (fq->paired ? 2 : 1); i++) {
            Input &in = fq->in[i];
            while (in.size - in.base < bytes && in.fill()) {
            }
        }
    } catch (...) {   // the next read meets the same condition itself
    }
}

}  // namespace
}  // namespace mica

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
            fq->in[i].f = fopen(i ? path2 : path1, "rb");
            if (!fq->in[i].f) return MICA_EIO;
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
    fq->join_ahead();
    try {
        // step 1: cut records (per file: the reads, or the mates, of the batch)
        const int files = fq->paired ? 2 : 1;
        const uint64_t want = fq->paired ? max_reads / 2 : max_reads;
        size_t pos[2] = {fq->in[0].base, fq->in[1].base};
        for (int i = 0; i < files; i++) {
            fq->spans[i].clear();
            if (int rc = cut_records(fq->in[i], &pos[i], want, fq->spans[i])) return rc;
        }
        if (fq->paired && fq->spans[0].size() != fq->spans[1].size()) return MICA_EIO;   // mate files differ
        const uint64_t n_rec = fq->spans[0].size();
        // step 2: check and pack chunks of records on host threads
        const uint64_t n_chunks = (n_rec + CHUNK_RECORDS - 1) / CHUNK_RECORDS;
        std::vector<Part> parts(n_chunks);
        Input *const in[2] = {&fq->in[0], &fq->in[1]};
        const uint64_t first = fq->next_read;
        parallel_chunks(n_chunks, host_threads(), [&](uint64_t c) {
            try {
                pack_chunk(parts[c], in, fq->spans, fq->paired, c * CHUNK_RECORDS,
                           std::min(n_rec, (c + 1) * CHUNK_RECORDS), first);
            } catch (const std::bad_alloc &) {
                parts[c].err = MICA_ENOMEM;
            }
        });
        for (const Part &p : parts)   // the first bad record in file order decides
            if (p.err) return p.err;
        std::unique_ptr<mica_read_batch> b(new mica_read_batch());
        b->paired = fq->paired;
        join_parts(*b, parts, k);
        size_t used = 0;
        for (int i = 0; i < files; i++) {
            used = std::max(used, pos[i] - fq->in[i].base);
            fq->in[i].consume(pos[i]);
        }
        fq->next_read += b->n();
        if (b->n() == max_reads) {   // likely more to come: read its bytes ahead
            try {
                fq->ahead = std::thread(read_ahead, fq, std::min<size_t>(used, size_t(1) << 30));
            } catch (const std::system_error &) {
            }
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
        // decided (reads in chunks on host threads) before anything changes
        const uint64_t base0 = offsets[0];
        std::vector<uint8_t> dn(offsets[n] - base0, 0xffu);
        const uint64_t chunk = 16384, n_chunks = (n + chunk - 1) / chunk;
        std::atomic<bool> bad{false};
        parallel_chunks(n_chunks, host_threads(), [&](uint64_t c) {
            uint8_t codes[MICA_MAX_READ_LEN], amb[MICA_MAX_READ_LEN];
            for (uint64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); i++) {
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
                    if (x.strand > 1 || x.pos >= text_len || m > text_len - x.pos) {
                        bad = true;
                        continue;
                    }
                    uint32_t raw = 0, dprime = 0;
                    for (uint32_t j = 0; j < m; j++) {
                        const uint32_t ri = x.strand ? m - 1 - j : j;   // read offset at window offset j
                        const uint8_t base = x.strand ? (uint8_t)(3 - codes[ri]) : codes[ri];
                        const bool mism = ref->text[x.pos + j] != (uint8_t)"ACGT"[base];
                        raw += mism;
                        dprime += mism || amb[ri];
                    }
                    if (x.mm != raw && x.mm != dprime) bad = true;
                    dn[h - base0] = (uint8_t)std::min<uint32_t>(dprime, 0xfeu);
                }
            }
        });
        if (bad) return MICA_EINVAL;
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
