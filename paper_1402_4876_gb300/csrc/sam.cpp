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
// input leaves the file as it was.  Records are independent per read (per
// pair), so both the check and the formatting run on host threads over
// chunks of 4,096 reads; formatted chunks are written in read order.
#include <algorithm>
#include <atomic>
#include <cstdio>
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

// Formatted records of one chunk: bytes [0, n) of data.  Room for a whole
// record is made before it is written (begin), so the writes themselves go
// through a plain cursor.
struct Out {
    std::vector<char> data;
    size_t n = 0;
    char *p = nullptr;

    void begin(size_t room)
    {
        if (data.size() < n + room) data.resize(std::max(n + room, 2 * data.size()));
        p = data.data() + n;
    }
    void end() { n = (size_t)(p - data.data()); }
    void put(char c) { *p++ = c; }
    void put(const char *s, size_t len)
    {
        memcpy(p, s, len);
        p += len;
    }
    template <size_t L> void lit(const char (&s)[L]) { put(s, L - 1); }
    void put(const std::string &s) { put(s.data(), s.size()); }
    void u64(uint64_t v)
    {
        char t[24];
        int k = 0;
        do {
            t[k++] = (char)('0' + v % 10);
            v /= 10;
        } while (v);
        while (k) *p++ = t[--k];
    }
    void i64(int64_t v)
    {
        if (v < 0) {
            put('-');
            u64((uint64_t)(-(v + 1)) + 1);
        } else {
            u64((uint64_t)v);
        }
    }
};

}  // namespace mica

struct mica_sam_writer {
    FILE *f = nullptr;
    const mica_reference *ref = nullptr;
    std::string prefix;
    uint32_t secondary = 0;
    uint32_t threads = 1;
    uint64_t next_id = 0;          // number of the next read, or of the next pair
    std::vector<mica::Out> bufs;   // one per chunk of a formatting window, kept across calls
    size_t name_room = 0;          // the longest contig name
};

namespace mica {
namespace {

constexpr const char *ACGT = "ACGT";
constexpr uint64_t CHUNK_READS = 4096;   // even: a pair never straddles two chunks

struct Placement {
    const mica_hit *h;
    int32_t contig;
    uint32_t local;   // 0-based coordinate in the contig
    uint32_t d;       // substitutions, ambiguous read bases included
};

// One read of the batch as the records need it.
struct ReadInfo {
    uint32_t m = 0;
    // the read as the window of a hit on strand s reads it: bases[s][j] is
    // the base at window offset j ('A'..'T', stand-ins for ambiguous bases)
    // and ambo[s][j] = 1 where that base is ambiguous (a substitution
    // wherever it falls); s = 1 is the reverse complement
    char bases[2][MICA_MAX_READ_LEN + 16];   // + room for whole-word decoding
    uint8_t ambo[2][MICA_MAX_READ_LEN];
    bool has_amb = false;
    bool ambo_clear = false;   // ambo holds zeros for the whole read length
    const char *name = nullptr;       // from a read batch, else NULL
    const char *qual = nullptr;
    uint64_t b = 0, e = 0;          // listed hits [b, e)
    std::vector<Placement> V;       // listed hits that are placements on the reference
    const Placement *primary = nullptr;
    uint32_t dmin = 0;
    uint64_t c0 = 0, c1 = 0;        // |V| at dmin, at dmin + 1
    bool complete = false;          // every hit listed
    int mapq = 0;
    uint64_t total_ref = 0;
};

// The four bases of one byte of a packed word (least significant first) as
// ASCII, and their complements in reverse order, four bytes each.
struct DecodeTable {
    char fwd[256][4], rc[256][4];
    DecodeTable()
    {
        for (int v = 0; v < 256; v++)
            for (int t = 0; t < 4; t++) {
                const int c = (v >> (2 * t)) & 3;
                fwd[v][t] = ACGT[c];
                rc[v][3 - t] = ACGT[3 - c];
            }
    }
};
const DecodeTable DECODE;

// Substitutions of the read on `strand` against G[pos, pos + m): *raw counts
// the stand-in bases as bases, *dprime counts every ambiguous base.
void substitutions(const mica_reference &ref, const ReadInfo &r, uint64_t pos, int strand, uint32_t *raw,
                   uint32_t *dprime)
{
    const uint8_t *t = ref.text.data() + pos;
    const char *s = r.bases[strand];
    const uint8_t *am = r.ambo[strand];
    uint32_t a = 0, b = 0;
    for (uint32_t j = 0; j < r.m; j++) {
        const uint32_t mism = t[j] != (uint8_t)s[j];
        a += mism;
        b += mism | am[j];
    }
    *raw = a;
    *dprime = b;
}

// A batch as the writer receives it; rb (optional) adds names, qualities,
// ambiguous bases and budgets.
struct Batch {
    const uint32_t *words;
    const uint64_t *word_off;
    const uint16_t *len;
    const uint64_t *total;
    const uint64_t *offsets;
    const mica_hit *hits;
    const mica_pair *pairs;   // pairing rows, or NULL
    uint64_t n;
    const mica_read_batch *rb;
    bool paired;              // reads 2i and 2i + 1 are mates
};

// Decode and classify read i; `check` also recomputes every listed hit's
// substitutions against G.  Returns MICA_EINVAL on inconsistent input.
int classify(const mica_reference &ref, const Batch &bt, uint64_t i, bool check, ReadInfo &r)
{
    const uint64_t *word_off = bt.word_off, *total = bt.total, *offsets = bt.offsets;
    const mica_hit *hits = bt.hits;
    r.m = bt.len[i];
    if (r.m == 0 || r.m > MICA_MAX_READ_LEN || word_off[i + 1] < word_off[i] ||
        word_off[i + 1] - word_off[i] < (r.m + 15u) / 16u)
        return MICA_EINVAL;
    const uint32_t *w = bt.words + word_off[i];
    const uint32_t m = r.m;
    // forward: 4 bases per byte; reverse complement: the same bytes from
    // the last base backwards (written right to left into a padded array)
    const uint32_t nbytes = (m + 3) / 4;
    char *rc_end = r.bases[1] + 4 * nbytes;   // rc of bases [0, 4 * nbytes), its last 4*nbytes - m are padding
    for (uint32_t q = 0; q < nbytes; q++) {
        const uint8_t byte = (uint8_t)(w[q >> 2] >> (8 * (q & 3)));
        memcpy(r.bases[0] + 4 * q, DECODE.fwd[byte], 4);
        memcpy(rc_end - 4 * (q + 1), DECODE.rc[byte], 4);
    }
    // the rc of the padded read starts with 4 * nbytes - m padding bases
    if (4 * nbytes != m) memmove(r.bases[1], r.bases[1] + (4 * nbytes - m), m);
    if (!r.ambo_clear || r.has_amb) {
        memset(r.ambo[0], 0, MICA_MAX_READ_LEN);
        memset(r.ambo[1], 0, MICA_MAX_READ_LEN);
        r.ambo_clear = true;
    }
    r.has_amb = false;
    uint32_t kmax = MICA_MAX_K;
    if (bt.rb) {
        const mica_read_batch &rb = *bt.rb;
        for (uint64_t a = rb.amb_off[i]; a < rb.amb_off[i + 1]; a++) {
            r.ambo[0][rb.amb[a]] = 1;
            r.ambo[1][m - 1 - rb.amb[a]] = 1;
        }
        r.has_amb = rb.amb_off[i + 1] > rb.amb_off[i];
        if (r.has_amb) r.ambo_clear = false;
        r.name = rb.names.c_str() + rb.name_off[i];
        r.qual = rb.quals.data() + rb.qual_off[i];
        kmax = rb.k[i];
    }
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
        uint32_t raw = x.mm, d = x.mm;
        if (check || r.has_amb) {
            substitutions(ref, r, x.pos, x.strand, &raw, &d);
            // as the search gave it (raw), or after the N filter (d')
            if (check && x.mm != raw && !(r.has_amb && x.mm == d)) return MICA_EINVAL;
            if (!r.has_amb) d = raw;
        }
        if (c >= 0 && d <= kmax) r.V.push_back({&x, c, (uint32_t)(x.pos - ref.start[c]), d});
    }
    for (const Placement &p : r.V) dmin = std::min(dmin, p.d);
    for (uint64_t h = r.b; h < r.e; h++) {   // the cap cuts the search's highest d first
        uint32_t raw = hits[h].mm, dd = raw;
        if (r.has_amb) substitutions(ref, r, hits[h].pos, hits[h].strand, &raw, &dd);
        deeper0 |= raw > dmin;
        deeper1 |= raw > dmin + 1;
    }
    r.dmin = dmin;
    r.c0 = r.c1 = 0;
    for (const Placement &p : r.V) {
        if (p.d == dmin) {
            if (!r.primary) r.primary = &p;
            r.c0++;
        } else if (p.d == dmin + 1) {
            r.c1++;
        }
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

void put_md(Out &o, const mica_reference &ref, const ReadInfo &r, uint64_t pos, int strand)
{
    const uint8_t *t = ref.text.data() + pos;
    const char *s = r.bases[strand];
    const uint8_t *am = r.ambo[strand];
    uint64_t run = 0;
    for (uint32_t j = 0; j < r.m;) {
        if (!r.has_amb && j + 8 <= r.m) {   // eight matching bases at a time
            uint64_t x, y;
            memcpy(&x, t + j, 8);
            memcpy(&y, s + j, 8);
            if (x == y) {
                run += 8;
                j += 8;
                continue;
            }
        }
        if (!am[j] && t[j] == (uint8_t)s[j]) {
            run++;
        } else {
            o.u64(run);
            o.put((char)t[j]);
            run = 0;
        }
        j++;
    }
    o.u64(run);
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

// Formats records into one chunk's Out.
struct Formatter {
    Out &out;
    const mica_reference &ref;
    const std::string &prefix;
    bool secondary;
    size_t name_room;   // the longest contig name

    // An upper bound on one record's bytes: QNAME, two contig names, SEQ,
    // QUAL, MD (at most 4 bytes per base and a run) and the fixed fields.
    size_t room(const ReadInfo &r) const
    {
        const size_t qn = r.name ? strlen(r.name) : prefix.size() + 20;
        return qn + 2 * name_room + 6 * (size_t)r.m + 320;
    }

    void qname(uint64_t id, const ReadInfo &r)
    {
        if (r.name) {
            out.put(r.name, strlen(r.name));
        } else {
            out.put(prefix);
            out.u64(id);
        }
        out.put('\t');
    }

    void rname(int32_t contig)
    {
        if (contig < 0) out.put('*');
        else out.put(ref.names[contig]);
        out.put('\t');
    }

    // RNEXT and PNEXT of a record at contig `self` whose mate sits at `mate`.
    void next(int32_t self, const Spot *mate)
    {
        if (!mate || mate->contig < 0) {
            out.lit("*\t0\t");
            return;
        }
        if (mate->contig == self) out.put('=');
        else out.put(ref.names[mate->contig]);
        out.put('\t');
        out.u64(mate->pos1);
        out.put('\t');
    }

    // SEQ and QUAL on the forward strand of the reference
    void seq(const ReadInfo &r, int strand)
    {
        char *d = out.p;
        out.put(r.bases[strand], r.m);
        if (r.has_amb)
            for (uint32_t j = 0; j < r.m; j++)
                if (r.ambo[strand][j]) d[j] = 'N';
        out.put('\t');
        if (!r.qual) {
            out.put('*');
            return;
        }
        if (strand == 0) {
            out.put(r.qual, r.m);
        } else {
            for (uint32_t j = 0; j < r.m; j++) out.p[j] = r.qual[r.m - 1 - j];
            out.p += r.m;
        }
    }

    void match_tags(const ReadInfo &r, const Placement &p)
    {
        out.lit("\tNM:i:");
        out.u64(p.d);
        out.lit("\tMD:Z:");
        put_md(out, ref, r, p.h->pos, p.h->strand);
    }

    // One primary record.  flag0: the pairing bits; mate = NULL for single reads.
    void primary(uint64_t id, uint32_t flag0, const ReadInfo &r, const Placement *p, int mapq, const Spot &self,
                 const Spot *mate, int64_t tlen)
    {
        const uint32_t flag = flag0 | (p ? 0u : 4u) | (p && p->h->strand ? 16u : 0u);
        out.begin(room(r));
        qname(id, r);
        out.u64(flag);
        out.put('\t');
        rname(self.contig);
        out.u64(self.pos1);
        out.put('\t');
        out.u64(p ? (uint64_t)mapq : 0u);
        out.put('\t');
        if (p) {
            out.u64(r.m);
            out.lit("M\t");
        } else {
            out.lit("*\t");
        }
        next(self.contig, mate);
        out.i64(tlen);
        out.put('\t');
        seq(r, p ? p->h->strand : 0);
        if (p) {
            match_tags(r, *p);
            out.lit("\tX0:i:");
            out.u64(r.c0);
            out.lit("\tX1:i:");
            out.u64(r.c1);
            out.lit("\tZT:i:");
            out.u64(r.total_ref);
        }
        out.put('\n');
        out.end();
    }

    void secondaries(uint64_t id, uint32_t flag0, const ReadInfo &r, const Placement *p, const Spot *mate)
    {
        if (!secondary) return;
        for (const Placement &s : r.V) {
            if (&s == p) continue;
            out.begin(room(r));
            qname(id, r);
            out.u64(flag0 | 256u | (s.h->strand ? 16u : 0u));
            out.put('\t');
            rname(s.contig);
            out.u64((uint64_t)s.local + 1);
            out.lit("\t0\t");
            out.u64(r.m);
            out.lit("M\t");
            next(s.contig, mate);
            out.lit("0\t*\t*");
            match_tags(r, s);
            out.put('\n');
            out.end();
        }
    }
};

// Proper-pair placement of a pair: sets the two primaries and their MAPQ.
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

inline int classify_read(const mica_reference &ref, const Batch &b, uint64_t i, bool check, ReadInfo &r)
{
    return classify(ref, b, i, check, r);
}

// Checks reads [a, e) of the batch (a even when paired).
int check_range(const mica_reference &ref, const Batch &b, uint64_t a, uint64_t e, ReadInfo &r1, ReadInfo &r2)
{
    for (uint64_t i = a; i < e; i++) {
        ReadInfo &r = ((i - a) & 1) ? r2 : r1;
        if (int rc = classify_read(ref, b, i, true, r)) return rc;
        if (b.pairs && ((i - a) & 1)) {
            const Placement *p1 = nullptr, *p2 = nullptr;
            int mapq = 0;
            bool proper = false;
            if (int rc = proper_pair(b.pairs[i / 2], r1, r2, b.hits, &p1, &p2, &mapq, &proper)) return rc;
        }
    }
    return 0;
}

// Formats reads [a, e) of a checked batch; first_id = number of read a (of
// its pair when paired).
void format_range(Formatter &out, const Batch &b, uint64_t a, uint64_t e, uint64_t first_id, ReadInfo &r1,
                  ReadInfo &r2)
{
    const mica_reference &ref = out.ref;
    if (!b.paired) {
        for (uint64_t i = a; i < e; i++) {
            classify_read(ref, b, i, false, r1);
            const uint64_t id = first_id + (i - a);
            out.primary(id, 0, r1, r1.primary, r1.mapq, spot_of(r1.primary), nullptr, 0);
            out.secondaries(id, 0, r1, r1.primary, nullptr);
        }
        return;
    }
    for (uint64_t i = a; i < e; i += 2) {
        classify_read(ref, b, i, false, r1);
        classify_read(ref, b, i + 1, false, r2);
        const Placement *p1 = r1.primary, *p2 = r2.primary;
        int q1 = r1.mapq, q2 = r2.mapq, qp = 0;
        bool proper = false;
        const Placement *x = nullptr, *y = nullptr;
        if (b.pairs) proper_pair(b.pairs[i / 2], r1, r2, b.hits, &x, &y, &qp, &proper);
        if (proper) {
            p1 = x;
            p2 = y;
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
        const uint64_t id = first_id + (i - a) / 2;
        out.primary(id, f1, r1, p1, q1, s1, &s2, t1);
        out.secondaries(id, f1 & ~2u, r1, p1, &s2);
        out.primary(id, f2, r2, p2, q2, s2, &s1, t2);
        out.secondaries(id, f2 & ~2u, r2, p2, &s1);
    }
}

inline void set_error(std::atomic<int> &err, int rc)
{
    int none = 0;
    err.compare_exchange_strong(none, rc);
}

// Checks a whole batch, then formats and writes it (see mica_sam_write).
int write_records(mica_sam_writer *w, const Batch &b)
{
    const mica_reference &ref = *w->ref;
    const uint64_t n_reads = b.n;
    const bool pairs = b.paired;
    const uint64_t n_chunks = (n_reads + CHUNK_READS - 1) / CHUNK_READS;
    std::atomic<int> err{0};
    // pass 1: check everything, write nothing
    parallel_chunks(n_chunks, w->threads, [&](uint64_t c) {
        try {
            ReadInfo r1, r2;
            const uint64_t a = c * CHUNK_READS, e = std::min(n_reads, a + CHUNK_READS);
            if (int rc = check_range(ref, b, a, e, r1, r2)) set_error(err, rc);
        } catch (const std::bad_alloc &) {
            set_error(err, MICA_ENOMEM);
        }
    });
    if (int rc = err.load()) return rc;
    // pass 2: format windows of chunks in parallel into one half of a double
    // buffer while a writer thread writes the previous window from the other
    try {
        const uint64_t window = (uint64_t)w->threads * 4;
        if (w->bufs.size() < 2 * window) w->bufs.resize(2 * window);
        std::thread writer;
        std::atomic<bool> write_ok{true};
        auto write_window = [&](uint64_t half, uint64_t nw) {
            for (uint64_t j = 0; j < nw; j++) {
                const Out &o = w->bufs[half * window + j];
                if (fwrite(o.data.data(), 1, o.n, w->f) != o.n) {
                    write_ok = false;
                    return;
                }
            }
        };
        auto join_writer = [&]() {
            if (writer.joinable()) writer.join();
        };
        for (uint64_t c0 = 0, k = 0; c0 < n_chunks; c0 += window, k++) {
            const uint64_t nw = std::min(window, n_chunks - c0), half = k & 1;
            parallel_chunks(nw, w->threads, [&](uint64_t j) {
                try {
                    ReadInfo r1, r2;
                    const uint64_t a = (c0 + j) * CHUNK_READS, e = std::min(n_reads, a + CHUNK_READS);
                    Out &o = w->bufs[half * window + j];
                    o.n = 0;
                    Formatter out{o, ref, w->prefix, w->secondary != 0, w->name_room};
                    format_range(out, b, a, e, w->next_id + (pairs ? a / 2 : a), r1, r2);
                } catch (const std::bad_alloc &) {
                    set_error(err, MICA_ENOMEM);
                }
            });
            join_writer();
            if (!write_ok) return MICA_EIO;
            if (int rc = err.load()) return rc;
            try {
                writer = std::thread(write_window, half, nw);
            } catch (const std::system_error &) {
                write_window(half, nw);   // no thread to spare: write here
            }
        }
        join_writer();
        if (!write_ok) return MICA_EIO;
    } catch (const std::bad_alloc &) {
        return MICA_ENOMEM;
    }
    if (!b.rb) w->next_id += pairs ? n_reads / 2 : n_reads;
    return 0;
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
    p->threads = 0;
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
    if (prefix.size() > 200 || p.secondary > 1 || p.threads > MAX_HOST_THREADS) return MICA_EINVAL;
    for (char c : prefix)   // QNAME: printable, no '@'
        if ((unsigned char)c < 33 || (unsigned char)c > 126 || c == '@') return MICA_EINVAL;
    if (p.command_line && strpbrk(p.command_line, "\t\n\r")) return MICA_EINVAL;
    try {
        std::unique_ptr<mica_sam_writer> w(new mica_sam_writer());
        w->ref = ref;
        w->prefix = prefix;
        w->secondary = p.secondary;
        w->threads = p.threads ? p.threads : host_threads();
        for (const std::string &name : ref->names) w->name_room = std::max(w->name_room, name.size());
        std::string s = "@HD\tVN:1.6\tSO:unsorted\n";
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
        w->f = fopen(path, "wb");
        if (!w->f) return MICA_EIO;
        if (fwrite(s.data(), 1, s.size(), w->f) != s.size()) {
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
    return write_records(w, Batch{packed_reads, word_offsets, lengths, total, offsets, hits, pairs, n_reads, nullptr,
                                  pairs != nullptr});
}

int mica_sam_write_batch(mica_sam_writer *w, const mica_read_batch *b, const uint64_t *total,
                         const uint64_t *offsets, const mica_hit *hits, const mica_pair *pairs)
{
    if (!w || !b) return MICA_EINVAL;
    const uint64_t n = b->n();
    if (n == 0) return 0;
    if (!total || !offsets || (pairs && !b->paired)) return MICA_EINVAL;
    return write_records(w, Batch{b->words.data(), b->word_off.data(), b->len.data(), total, offsets, hits, pairs, n, b,
                                  b->paired});
}

int mica_sam_close(mica_sam_writer *w)
{
    if (!w) return MICA_EINVAL;
    const bool ok = fclose(w->f) == 0;
    delete w;
    return ok ? 0 : MICA_EIO;
}

}  // extern "C"
