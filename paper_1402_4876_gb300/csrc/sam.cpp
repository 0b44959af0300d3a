// SAM 1.6 output of the search's placements (host-side, no CUDA).  The paper's
// BWT phase places each read with few substitutions and passes the result on
// to SAM-producing stages (Section 2); this writer turns a result of the
// library (per read: exact total, listed hits sorted by position and strand)
// into SAM records against a mica_reference: contig names and 1-based
// coordinates, SEQ on the forward strand, CIGAR of matches only (the BWT
// phase allows no gaps), NM/MD recomputed against the reference text, a
// uniqueness MAPQ and, for paired reads, the pairing fields.
//
// A batch is checked in full before any of it is formatted, so that bad
// input leaves the file as it was.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "reference_internal.h"

struct mica_sam_writer {
    FILE *f = nullptr;
    const mica_reference *ref = nullptr;
    std::string prefix;
    uint32_t secondary = 0;
    uint64_t next_id = 0;   // number of the next read, or of the next pair
    std::string buf;
};

namespace mica {
namespace {

constexpr const char *ACGT = "ACGT";
constexpr size_t FLUSH_BYTES = 8u << 20;

struct Placement {
    const mica_hit *h;
    int32_t contig;
    uint32_t local;   // 0-based coordinate in the contig
};

// One read of the batch as the records need it.
struct ReadInfo {
    uint32_t m = 0;
    uint8_t codes[MICA_MAX_READ_LEN];
    uint64_t b = 0, e = 0;          // listed hits [b, e)
    std::vector<Placement> V;       // listed hits that are placements on the reference
    const Placement *primary = nullptr;
    uint32_t dmin = 0;
    uint64_t c0 = 0, c1 = 0;        // |V| at dmin, at dmin + 1
    bool complete = false;          // every hit listed
    int mapq = 0;
    uint64_t total_ref = 0;
};

// The read's base on `strand` at offset j of the matched window (the reverse
// complement for the - strand).
inline uint8_t oriented(const ReadInfo &r, int strand, uint32_t j)
{
    return strand == 0 ? r.codes[j] : (uint8_t)(3 - r.codes[r.m - 1 - j]);
}

uint32_t substitutions(const mica_reference &ref, const ReadInfo &r, uint64_t pos, int strand)
{
    uint32_t d = 0;
    for (uint32_t j = 0; j < r.m; j++) d += ref.text[pos + j] != (uint8_t)ACGT[oriented(r, strand, j)];
    return d;
}

// Decode and classify read i; `check` also recomputes every listed hit's
// substitutions against G.  Returns MICA_EINVAL on inconsistent input.
int classify(const mica_reference &ref, const uint32_t *words, const uint64_t *word_off, const uint16_t *len,
             const uint64_t *total, const uint64_t *offsets, const mica_hit *hits, uint64_t i, bool check,
             ReadInfo &r)
{
    r.m = len[i];
    if (r.m == 0 || r.m > MICA_MAX_READ_LEN || word_off[i + 1] < word_off[i] ||
        word_off[i + 1] - word_off[i] < (r.m + 15u) / 16u)
        return MICA_EINVAL;
    const uint32_t *w = words + word_off[i];
    for (uint32_t j = 0; j < r.m; j++) r.codes[j] = (uint8_t)((w[j >> 4] >> (2 * (j & 15))) & 3);
    r.b = offsets[i];
    r.e = offsets[i + 1];
    if (r.e < r.b || r.e - r.b > total[i] || (r.e > r.b && !hits)) return MICA_EINVAL;
    r.V.clear();
    r.primary = nullptr;
    uint32_t dmin = 0xffu;
    bool deeper0 = false, deeper1 = false;
    for (uint64_t h = r.b; h < r.e; h++) {
        const mica_hit &x = hits[h];
        const int32_t c = reference_place(ref, x.pos, r.m);
        if (c == PLACE_OUT_OF_RANGE || x.strand > 1 || x.mm > MICA_MAX_K) return MICA_EINVAL;
        if (check && substitutions(ref, r, x.pos, x.strand) != x.mm) return MICA_EINVAL;
        if (c >= 0) {
            r.V.push_back({&x, c, (uint32_t)(x.pos - ref.start[c])});
            dmin = std::min<uint32_t>(dmin, x.mm);
        }
    }
    r.dmin = dmin;
    r.c0 = r.c1 = 0;
    for (const Placement &p : r.V) {
        if (p.h->mm == dmin) {
            if (!r.primary) r.primary = &p;
            r.c0++;
        } else if (p.h->mm == dmin + 1) {
            r.c1++;
        }
    }
    for (uint64_t h = r.b; h < r.e; h++) {   // the cap cuts the highest d first
        deeper0 |= hits[h].mm > dmin;
        deeper1 |= hits[h].mm > dmin + 1;
    }
    const uint64_t listed = r.e - r.b;
    r.complete = total[i] == listed;
    const bool unique = r.c0 == 1 && (r.complete || deeper0);
    r.mapq = !unique ? 0 : (r.c1 == 0 && (r.complete || deeper1)) ? 37 : 25;
    r.total_ref = total[i] - (listed - r.V.size());
    return 0;
}

// The placement in V of a listed hit (pos, strand): *found = whether it is
// listed at all; returns NULL when it is not, or is off the reference.
const Placement *find_hit(const ReadInfo &r, const mica_hit *hits, uint32_t pos, uint8_t strand, bool *found)
{
    *found = false;
    for (uint64_t h = r.b; h < r.e; h++)
        if (hits[h].pos == pos && hits[h].strand == strand) {
            *found = true;
            for (const Placement &p : r.V)
                if (p.h == hits + h) return &p;
            return nullptr;
        }
    return nullptr;
}

inline void put_u64(std::string &s, uint64_t v)
{
    char t[24];
    int n = 0;
    do {
        t[n++] = (char)('0' + v % 10);
        v /= 10;
    } while (v);
    while (n) s.push_back(t[--n]);
}

inline void put_i64(std::string &s, int64_t v)
{
    if (v < 0) {
        s.push_back('-');
        put_u64(s, (uint64_t)(-(v + 1)) + 1);
    } else {
        put_u64(s, (uint64_t)v);
    }
}

void put_md(std::string &s, const mica_reference &ref, const ReadInfo &r, uint64_t pos, int strand)
{
    uint64_t run = 0;
    for (uint32_t j = 0; j < r.m; j++) {
        const uint8_t g = ref.text[pos + j];
        if (g == (uint8_t)ACGT[oriented(r, strand, j)]) {
            run++;
        } else {
            put_u64(s, run);
            s.push_back((char)g);
            run = 0;
        }
    }
    put_u64(s, run);
}

// Where a read's primary record sits: its own primary placement, or (for an
// unmapped read with a mapped mate) the mate's; contig -1 = nowhere.
struct Spot {
    int32_t contig = -1;
    uint64_t pos1 = 0;
};

inline Spot spot_of(const Placement *p)
{
    Spot s;
    if (p) {
        s.contig = p->contig;
        s.pos1 = (uint64_t)p->local + 1;
    }
    return s;
}

struct Writer {
    mica_sam_writer &w;
    const mica_reference &ref;

    void qname(uint64_t id)
    {
        w.buf += w.prefix;
        put_u64(w.buf, id);
        w.buf.push_back('\t');
    }

    void rname(int32_t contig)
    {
        if (contig < 0) w.buf.push_back('*');
        else w.buf += ref.names[contig];
        w.buf.push_back('\t');
    }

    // RNEXT and PNEXT of a record at contig `self` whose mate sits at `mate`.
    void next(int32_t self, const Spot *mate)
    {
        if (!mate || mate->contig < 0) {
            w.buf += "*\t0\t";
            return;
        }
        if (mate->contig == self) w.buf.push_back('=');
        else w.buf += ref.names[mate->contig];
        w.buf.push_back('\t');
        put_u64(w.buf, mate->pos1);
        w.buf.push_back('\t');
    }

    void seq(const ReadInfo &r, int strand)
    {
        for (uint32_t j = 0; j < r.m; j++) w.buf.push_back(ACGT[oriented(r, strand, j)]);
        w.buf += "\t*";   // SEQ, QUAL
    }

    void match_tags(const ReadInfo &r, const Placement &p)
    {
        w.buf += "\tNM:i:";
        put_u64(w.buf, p.h->mm);
        w.buf += "\tMD:Z:";
        put_md(w.buf, ref, r, p.h->pos, p.h->strand);
    }

    // One primary record.  flag0: the pairing bits; mate = NULL for single reads.
    void primary(uint64_t id, uint32_t flag0, const ReadInfo &r, const Placement *p, int mapq, const Spot &self,
                 const Spot *mate, int64_t tlen)
    {
        const uint32_t flag = flag0 | (p ? 0u : 4u) | (p && p->h->strand ? 16u : 0u);
        qname(id);
        put_u64(w.buf, flag);
        w.buf.push_back('\t');
        rname(self.contig);
        put_u64(w.buf, self.pos1);
        w.buf.push_back('\t');
        put_u64(w.buf, p ? (uint64_t)mapq : 0u);
        w.buf.push_back('\t');
        if (p) {
            put_u64(w.buf, r.m);
            w.buf += "M\t";
        } else {
            w.buf += "*\t";
        }
        next(self.contig, mate);
        put_i64(w.buf, tlen);
        w.buf.push_back('\t');
        seq(r, p ? p->h->strand : 0);
        if (p) {
            match_tags(r, *p);
            w.buf += "\tX0:i:";
            put_u64(w.buf, r.c0);
            w.buf += "\tX1:i:";
            put_u64(w.buf, r.c1);
            w.buf += "\tZT:i:";
            put_u64(w.buf, r.total_ref);
        }
        w.buf.push_back('\n');
    }

    void secondaries(uint64_t id, uint32_t flag0, const ReadInfo &r, const Placement *p, const Spot *mate)
    {
        if (!w.secondary) return;
        for (const Placement &s : r.V) {
            if (&s == p) continue;
            qname(id);
            put_u64(w.buf, flag0 | 256u | (s.h->strand ? 16u : 0u));
            w.buf.push_back('\t');
            rname(s.contig);
            put_u64(w.buf, (uint64_t)s.local + 1);
            w.buf += "\t0\t";
            put_u64(w.buf, r.m);
            w.buf += "M\t";
            next(s.contig, mate);
            w.buf += "0\t*\t*";
            match_tags(r, s);
            w.buf.push_back('\n');
        }
    }
};

bool flush(mica_sam_writer &w)
{
    if (w.buf.empty()) return true;
    const bool ok = fwrite(w.buf.data(), 1, w.buf.size(), w.f) == w.buf.size();
    w.buf.clear();
    return ok;
}

// Proper-pair placement of pair i, or false.  Sets the two primaries and MAPQ.
int proper_pair(const mica_pair &pr, const ReadInfo &m1, const ReadInfo &m2, const mica_hit *hits,
                const Placement **p1, const Placement **p2, int *mapq, bool *proper)
{
    *proper = false;
    if (pr.n_concordant == 0) return 0;
    if (pr.plus_mate > 1) return MICA_EINVAL;
    const ReadInfo &plus = pr.plus_mate == 0 ? m1 : m2, &minus = pr.plus_mate == 0 ? m2 : m1;
    bool found_p = false, found_m = false;
    const Placement *a = find_hit(plus, hits, pr.pos_plus, 0, &found_p);
    const Placement *b = find_hit(minus, hits, pr.pos_minus, 1, &found_m);
    if (!found_p || !found_m) return MICA_EINVAL;   // the pairing does not belong to this result
    if (!a || !b || a->contig != b->contig) return 0;
    *p1 = pr.plus_mate == 0 ? a : b;
    *p2 = pr.plus_mate == 0 ? b : a;
    *mapq = pr.n_best > 1 ? 0 : (pr.n_concordant == 1 && m1.complete && m2.complete) ? 37 : 25;
    *proper = true;
    return 0;
}

// TLEN of mate `self` against `other` (both mapped in one contig), + on the
// mate that starts first, mate 1 on a tie.
int64_t tlen_of(const Placement &self, uint32_t mself, const Placement &other, uint32_t mother, bool self_is_mate1)
{
    const uint64_t s0 = self.local, s1 = other.local;
    const uint64_t lo = std::min(s0, s1), hi = std::max(s0 + mself, s1 + mother);
    const int64_t t = (int64_t)(hi - lo);
    if (s0 != s1) return s0 < s1 ? t : -t;
    return self_is_mate1 ? t : -t;
}

}  // namespace
}  // namespace mica

using namespace mica;

extern "C" {

void mica_sam_params_default(mica_sam_params *p)
{
    if (!p) return;
    p->qname_prefix = nullptr;
    p->secondary = 0;
    p->command_line = nullptr;
}

int mica_sam_open(const char *path, const mica_reference *ref, const mica_sam_params *params,
                  mica_sam_writer **out)
{
    if (!out) return MICA_EINVAL;
    *out = nullptr;
    if (!path || !ref) return MICA_EINVAL;
    mica_sam_params p;
    mica_sam_params_default(&p);
    if (params) p = *params;
    const std::string prefix = p.qname_prefix ? p.qname_prefix : "r";
    if (prefix.size() > 200 || p.secondary > 1) return MICA_EINVAL;
    for (char c : prefix)   // QNAME: printable, no '@'
        if ((unsigned char)c < 33 || (unsigned char)c > 126 || c == '@') return MICA_EINVAL;
    if (p.command_line && strpbrk(p.command_line, "\t\n\r")) return MICA_EINVAL;
    try {
        std::unique_ptr<mica_sam_writer> w(new mica_sam_writer());
        w->ref = ref;
        w->prefix = prefix;
        w->secondary = p.secondary;
        w->f = fopen(path, "wb");
        if (!w->f) return MICA_EIO;
        std::string &s = w->buf;
        s += "@HD\tVN:1.6\tSO:unsorted\n";
        for (size_t i = 0; i < ref->names.size(); i++) {
            s += "@SQ\tSN:";
            s += ref->names[i];
            s += "\tLN:";
            put_u64(s, ref->start[i + 1] - ref->start[i]);
            s.push_back('\n');
        }
        s += "@PG\tID:mica-gb300\tPN:mica-gb300\tVN:1.0";
        if (p.command_line) {
            s += "\tCL:";
            s += p.command_line;
        }
        s.push_back('\n');
        if (!flush(*w)) {
            fclose(w->f);
            return MICA_EIO;
        }
        *out = w.release();
        return 0;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
}

int mica_sam_write(mica_sam_writer *w, const uint32_t *packed_reads, const uint64_t *word_offsets,
                   const uint16_t *lengths, uint64_t n_reads, const uint64_t *total, const uint64_t *offsets,
                   const mica_hit *hits, const mica_pair *pairs)
{
    if (!w) return MICA_EINVAL;
    if (n_reads == 0) return 0;
    if (!packed_reads || !word_offsets || !lengths || !total || !offsets) return MICA_EINVAL;
    if (pairs && (n_reads & 1)) return MICA_EINVAL;
    const mica_reference &ref = *w->ref;
    try {
        ReadInfo r1, r2;
        // pass 1: check everything, write nothing
        for (uint64_t i = 0; i < n_reads; i++) {
            ReadInfo &r = (i & 1) ? r2 : r1;
            if (int rc = classify(ref, packed_reads, word_offsets, lengths, total, offsets, hits, i, true, r))
                return rc;
            if (pairs && (i & 1)) {
                const Placement *p1 = nullptr, *p2 = nullptr;
                int mapq = 0;
                bool proper = false;
                if (int rc = proper_pair(pairs[i / 2], r1, r2, hits, &p1, &p2, &mapq, &proper)) return rc;
            }
        }
        // pass 2: format
        Writer out{*w, ref};
        if (!pairs) {
            for (uint64_t i = 0; i < n_reads; i++) {
                classify(ref, packed_reads, word_offsets, lengths, total, offsets, hits, i, false, r1);
                const Spot self = spot_of(r1.primary);
                out.primary(w->next_id + i, 0, r1, r1.primary, r1.mapq, self, nullptr, 0);
                out.secondaries(w->next_id + i, 0, r1, r1.primary, nullptr);
                if (w->buf.size() >= FLUSH_BYTES && !flush(*w)) return MICA_EIO;
            }
            w->next_id += n_reads;
        } else {
            for (uint64_t i = 0; i < n_reads; i += 2) {
                classify(ref, packed_reads, word_offsets, lengths, total, offsets, hits, i, false, r1);
                classify(ref, packed_reads, word_offsets, lengths, total, offsets, hits, i + 1, false, r2);
                const Placement *p1 = r1.primary, *p2 = r2.primary;
                int q1 = r1.mapq, q2 = r2.mapq, qp = 0;
                bool proper = false;
                const Placement *a = nullptr, *b = nullptr;
                proper_pair(pairs[i / 2], r1, r2, hits, &a, &b, &qp, &proper);
                if (proper) {
                    p1 = a;
                    p2 = b;
                    q1 = q2 = qp;
                }
                // an unmapped mate sits at its mapped mate's place
                Spot s1 = spot_of(p1), s2 = spot_of(p2);
                if (!p1) s1 = s2;
                if (!p2) s2 = s1;
                int64_t t1 = 0, t2 = 0;
                if (p1 && p2 && p1->contig == p2->contig) {
                    t1 = tlen_of(*p1, r1.m, *p2, r2.m, true);
                    t2 = tlen_of(*p2, r2.m, *p1, r1.m, false);
                }
                const uint32_t base = 1u | (proper ? 2u : 0u);
                const uint32_t f1 = base | 64u | (p2 ? (p2->h->strand ? 32u : 0u) : 8u);
                const uint32_t f2 = base | 128u | (p1 ? (p1->h->strand ? 32u : 0u) : 8u);
                const uint64_t id = w->next_id + i / 2;
                out.primary(id, f1, r1, p1, q1, s1, &s2, t1);
                out.secondaries(id, f1 & ~2u, r1, p1, &s2);
                out.primary(id, f2, r2, p2, q2, s2, &s1, t2);
                out.secondaries(id, f2 & ~2u, r2, p2, &s1);
                if (w->buf.size() >= FLUSH_BYTES && !flush(*w)) return MICA_EIO;
            }
            w->next_id += n_reads / 2;
        }
        return flush(*w) ? 0 : MICA_EIO;
    } catch (const std::bad_alloc &) {
        w->buf.clear();
        return MICA_ENOMEM;
    }
}

int mica_sam_close(mica_sam_writer *w)
{
    if (!w) return MICA_EINVAL;
    bool ok = flush(*w);
    ok = fclose(w->f) == 0 && ok;
    delete w;
    return ok ? 0 : MICA_EIO;
}

}  // extern "C"
