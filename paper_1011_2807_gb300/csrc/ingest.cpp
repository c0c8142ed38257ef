// MS/MS spectra -> sparse vectors (Section 5's preprocessing), host code.
//
// Section 5 turns each spectrum into one sparse vector: every peak is a feature, its
// m/z multiplied by 10 is the dimension index and its intensity is the value.  This
// file reads the two plain-text peak-list formats such spectra come in and builds that
// CSR on the host:
//   - MGF: spectra between "BEGIN IONS" and "END IONS"; inside, KEY=VALUE header lines
//     (TITLE, PEPMASS, CHARGE, ...) and peak lines "m/z intensity [charge]";
//   - MS2: "H" lines (file header), then per spectrum an "S" line followed by "I", "Z"
//     or "D" lines and peak lines "m/z intensity".
// Lines may end in LF or CRLF; fields are separated by spaces or tabs; blank lines and
// lines starting with '#', ';' or '!' are comments.  Numbers are decimal or scientific
// (std::from_chars, correctly rounded and locale-free; a leading '+' is allowed).
//
// Large inputs are cut at spectrum starts (BEGIN IONS / S lines) into chunks that host
// threads parse side by side; the chunks' rows are then concatenated in file order, so
// the result, and the error reported for a malformed input (the first in file order,
// with its line number), are those of one sequential pass.
//
// Where the paper is silent (every choice below can be changed through knn_spectra_opts):
//   - the dimension is floor(m/z * mz_scale); a product within 2^-20 below an integer
//     counts as that integer, so that decimal m/z values whose binary value falls just
//     short (0.7 * 10 = 6.9999999999999996) land in the bin their digits name;
//   - peaks of one spectrum that fall in the same dimension keep the largest intensity
//     (the value is then still the intensity of one of its peaks), or their sum;
//   - peaks with intensity <= min_intensity (default 0) are dropped: a feature's
//     weight must be positive;
//   - uint8 weights, when asked for, are ceil(100 * I / I_max) with I_max the
//     spectrum's largest (merged) intensity: 1..100, the weight range of the
//     spectrum-shaped synthetic workload.
#include "knn_join.h"

#include <algorithm>
#include <cerrno>
#include <charconv>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <utility>
#include <vector>

namespace knn {
knn_status fail(knn_status st, const char* fmt, ...);
}

struct knn_spectra {
    std::vector<int64_t> indptr{0};
    std::vector<int32_t> indices;
    std::vector<float> values_f32;
    std::vector<uint8_t> values_u8;
    knn_dtype dtype = KNN_F32;
    int32_t dim = 0;
    knn_spectra_info info{};
};

namespace {

using knn::fail;

constexpr double BIN_SNAP = 1.0 / 1048576.0;   // 2^-20

struct Peak {
    int64_t d;
    double w;
};

struct Parser {
    const char* p;      // current position
    const char* end;
    int64_t line = 0;   // 1-based number (in the whole input) of the line last read
    const char* ls = nullptr;   // that line: [ls, le), without its line ending
    const char* le = nullptr;

    bool next_line() {
        if (p >= end) return false;
        ls = p;
        const char* nl = (const char*)memchr(p, '\n', (size_t)(end - p));
        le = nl ? nl : end;
        p = nl ? nl + 1 : end;
        if (le > ls && le[-1] == '\r') le--;
        line++;
        return true;
    }
};

inline bool is_space(char c) { return c == ' ' || c == '\t'; }

// [s, e) without leading and trailing blanks
inline void trim(const char*& s, const char*& e) {
    while (s < e && is_space(*s)) s++;
    while (e > s && is_space(e[-1])) e--;
}

inline bool is_comment_or_blank(const char* s, const char* e) {
    trim(s, e);
    return s == e || *s == '#' || *s == ';' || *s == '!';
}

// Case-insensitive equality of the trimmed line with `word`.
inline bool line_is(const char* s, const char* e, const char* word) {
    trim(s, e);
    const size_t n = strlen(word);
    if ((size_t)(e - s) != n) return false;
    for (size_t i = 0; i < n; i++) {
        char a = s[i], b = word[i];
        if (a >= 'a' && a <= 'z') a = (char)(a - 'a' + 'A');
        if (a != b) return false;
    }
    return true;
}

// Reads the number that starts the next field at s (after blanks) and moves s past it.
// Returns false if the field is missing or is not entirely a number.
inline bool read_number(const char*& s, const char* e, double* out) {
    while (s < e && is_space(*s)) s++;
    if (s >= e) return false;
    const char* t = s;
    while (t < e && !is_space(*t)) t++;
    const char* a = s;
    if (*a == '+' && t - a > 1 && *(a + 1) != '-' && *(a + 1) != '+') a++;
    double v = 0.0;
    const std::from_chars_result r = std::from_chars(a, t, v);
    if (r.ec == std::errc::result_out_of_range) {   // past double's range: infinity or a tiny value
        char buf[64];
        const size_t n = (size_t)(t - s);
        if (n + 1 > sizeof(buf)) return false;
        memcpy(buf, s, n);
        buf[n] = '\0';
        char* stop = nullptr;
        v = strtod(buf, &stop);
        if (stop != buf + n) return false;
    } else if (r.ec != std::errc() || r.ptr != t) {
        return false;
    }
    *out = v;
    s = t;
    return true;
}

}  // namespace

#define SPECTRA_TRY(expr)                     \
    do {                                      \
        const knn_status st_ = (expr);        \
        if (st_ != KNN_OK) return st_;        \
    } while (0)

namespace {

// Collects one spectrum's peaks at a time and appends it to the CSR when it ends.
struct Builder {
    const knn_spectra_opts& o;
    knn_spectra& out;
    std::vector<Peak> peaks;   // the open spectrum's kept peaks, in file order
    bool open = false;
    int64_t max_d = -1;

    Builder(const knn_spectra_opts& opts, knn_spectra& sp) : o(opts), out(sp) {}

    void begin() {
        peaks.clear();
        open = true;
    }

    knn_status add_peak(double mz, double inten, int64_t line) {
        if (!std::isfinite(mz) || mz < 0.0)
            return fail(KNN_EINVAL, "line %lld: m/z must be finite and >= 0", (long long)line);
        if (!std::isfinite(inten)) return fail(KNN_EINVAL, "line %lld: intensity is not finite", (long long)line);
        out.info.n_peaks++;
        if (!(inten > o.min_intensity)) {
            out.info.n_dropped++;
            return KNN_OK;
        }
        const double x = mz * o.mz_scale;   // Section 5: m/z times 10 is the dimension index
        double fl = std::floor(x);
        if (x - fl >= 1.0 - BIN_SNAP) fl += 1.0;
        if (fl > 2147483646.0)
            return fail(KNN_EUNSUPPORTED, "line %lld: dimension %.0f does not fit int32", (long long)line, fl);
        const int64_t d = (int64_t)fl;
        if (o.dim > 0 && d >= o.dim)
            return fail(KNN_EINVAL, "line %lld: m/z %.17g gives dimension %lld, not below dim = %d", (long long)line,
                        mz, (long long)d, o.dim);
        peaks.push_back({d, inten});
        return KNN_OK;
    }

    knn_status end_spectrum() {
        // ascending dimension; file order within a dimension (the order of a sum)
        std::stable_sort(peaks.begin(), peaks.end(), [](const Peak& a, const Peak& b) { return a.d < b.d; });
        size_t m = 0;
        for (size_t i = 0; i < peaks.size();) {
            double w = peaks[i].w;
            size_t j = i + 1;
            for (; j < peaks.size() && peaks[j].d == peaks[i].d; j++) {
                w = o.merge == KNN_MERGE_SUM ? w + peaks[j].w : std::max(w, peaks[j].w);
                out.info.n_merged++;
            }
            peaks[m++] = {peaks[i].d, w};
            i = j;
        }
        peaks.resize(m);
        if (o.weights == KNN_SPECTRA_U8) {
            double imax = 0.0;
            for (const Peak& q : peaks) imax = std::max(imax, q.w);
            for (const Peak& q : peaks) {
                double c = std::ceil(100.0 * q.w / imax);
                c = std::min(100.0, std::max(1.0, c));
                out.indices.push_back((int32_t)q.d);
                out.values_u8.push_back((uint8_t)c);
                max_d = std::max(max_d, q.d);
            }
        } else {
            for (const Peak& q : peaks) {
                const float f = (float)q.w;
                if (std::isinf(f)) return fail(KNN_EUNSUPPORTED, "an intensity of %.17g does not fit float32", q.w);
                if (!(f > 0.0f)) {   // below float32's smallest positive value
                    out.info.n_dropped++;
                    continue;
                }
                out.indices.push_back((int32_t)q.d);
                out.values_f32.push_back(f);
                max_d = std::max(max_d, q.d);
            }
        }
        out.indptr.push_back((int64_t)out.indices.size());
        out.info.n_spectra++;
        open = false;
        return KNN_OK;
    }
};

// `last`: the chunk runs to the end of the input; otherwise the next chunk starts with
// a BEGIN IONS line, which is where a spectrum still open here is reported.
knn_status parse_mgf(Parser& ps, Builder& b, bool last) {
    while (ps.next_line()) {
        const char *s = ps.ls, *e = ps.le;
        if (is_comment_or_blank(s, e)) continue;
        if (!b.open) {
            if (line_is(s, e, "BEGIN IONS")) b.begin();
            else if (line_is(s, e, "END IONS"))
                return fail(KNN_EINVAL, "line %lld: END IONS without BEGIN IONS", (long long)ps.line);
            continue;   // file-level parameters (KEY=VALUE) between spectra
        }
        if (line_is(s, e, "END IONS")) {
            SPECTRA_TRY(b.end_spectrum());
            continue;
        }
        if (line_is(s, e, "BEGIN IONS"))
            return fail(KNN_EINVAL, "line %lld: BEGIN IONS inside a spectrum", (long long)ps.line);
        trim(s, e);
        if ((*s >= 'A' && *s <= 'Z') || (*s >= 'a' && *s <= 'z')) {   // TITLE=..., PEPMASS=..., CHARGE=...
            if (!memchr(s, '=', (size_t)(e - s)))
                return fail(KNN_EINVAL, "line %lld: neither a KEY=VALUE header nor a peak", (long long)ps.line);
            continue;
        }
        double mz = 0.0, in = 0.0;
        if (!read_number(s, e, &mz) || !read_number(s, e, &in))
            return fail(KNN_EINVAL, "line %lld: a peak line needs an m/z and an intensity", (long long)ps.line);
        SPECTRA_TRY(b.add_peak(mz, in, ps.line));   // a third field (fragment charge) is ignored
    }
    if (b.open) {
        if (!last) return fail(KNN_EINVAL, "line %lld: BEGIN IONS inside a spectrum", (long long)(ps.line + 1));
        return fail(KNN_EINVAL, "the input ends inside a spectrum (no END IONS)");
    }
    return KNN_OK;
}

knn_status parse_ms2(Parser& ps, Builder& b) {
    while (ps.next_line()) {
        const char *s = ps.ls, *e = ps.le;
        if (is_comment_or_blank(s, e)) continue;
        trim(s, e);
        const char c = *s;
        if ((c >= 'A' && c <= 'Z') || (c >= 'a' && c <= 'z')) {
            if (e - s > 1 && !is_space(s[1]))
                return fail(KNN_EINVAL, "line %lld: a record type is one letter", (long long)ps.line);
            if (c == 'S') {   // a new spectrum: S <first scan> <last scan> <precursor m/z>
                if (b.open) SPECTRA_TRY(b.end_spectrum());
                b.begin();
            } else if (c == 'H') {
                if (b.open || b.out.info.n_spectra > 0)
                    return fail(KNN_EINVAL, "line %lld: H line after the first spectrum", (long long)ps.line);
            } else if (c == 'I' || c == 'Z' || c == 'D') {
                if (!b.open) return fail(KNN_EINVAL, "line %lld: %c line before the first S line", (long long)ps.line, c);
            } else {
                return fail(KNN_EINVAL, "line %lld: unknown record type '%c'", (long long)ps.line, c);
            }
            continue;
        }
        if (!b.open) return fail(KNN_EINVAL, "line %lld: a peak before the first S line", (long long)ps.line);
        double mz = 0.0, in = 0.0;
        if (!read_number(s, e, &mz) || !read_number(s, e, &in))
            return fail(KNN_EINVAL, "line %lld: a peak line needs an m/z and an intensity", (long long)ps.line);
        SPECTRA_TRY(b.add_peak(mz, in, ps.line));
    }
    if (b.open) SPECTRA_TRY(b.end_spectrum());
    return KNN_OK;
}

// MGF if the first line that is not a comment is BEGIN IONS or a KEY=VALUE parameter;
// MS2 if it is a one-letter H or S record; MGF (no spectra) if every line is a comment.
knn_spectra_format detect(const char* text, size_t len) {
    Parser ps{text, text + len};
    while (ps.next_line()) {
        const char *s = ps.ls, *e = ps.le;
        if (is_comment_or_blank(s, e)) continue;
        trim(s, e);
        if (line_is(s, e, "BEGIN IONS") || memchr(s, '=', (size_t)(e - s))) return KNN_SPECTRA_MGF;
        if ((*s == 'H' || *s == 'S') && (e - s == 1 || is_space(s[1]))) return KNN_SPECTRA_MS2;
        return KNN_SPECTRA_AUTO;
    }
    return KNN_SPECTRA_MGF;
}

// Whether the line [s, e) starts a spectrum of format fmt.
bool starts_spectrum(const char* s, const char* e, knn_spectra_format fmt) {
    if (e > s && e[-1] == '\r') e--;
    if (fmt == KNN_SPECTRA_MGF) return line_is(s, e, "BEGIN IONS");
    trim(s, e);
    return s < e && *s == 'S' && (e - s == 1 || is_space(s[1]));
}

// Chunk boundaries cut[0] = 0 <= cut[1] <= ... <= cut[T] = len: each inner one is the
// start of the first line at or after c * len / T that starts a spectrum (len if none).
std::vector<size_t> split_points(const char* text, size_t len, knn_spectra_format fmt, int T) {
    std::vector<size_t> cut((size_t)T + 1, 0);
    cut[(size_t)T] = len;
    for (int c = 1; c < T; c++) {
        size_t q = std::max(cut[(size_t)c - 1], (size_t)((double)len * c / T));
        if (q > 0 && q < len && text[q - 1] != '\n') {   // to the next line start
            const char* nl = (const char*)memchr(text + q, '\n', len - q);
            q = nl ? (size_t)(nl - text) + 1 : len;
        }
        while (q < len) {
            const char* nl = (const char*)memchr(text + q, '\n', len - q);
            const size_t le = nl ? (size_t)(nl - text) : len;
            if (starts_spectrum(text + q, text + le, fmt)) break;
            q = nl ? le + 1 : len;
        }
        cut[(size_t)c] = std::min(q, len);
    }
    return cut;
}

// Runs f(0..n-1), on n threads when n > 1.
template <class F>
void run_parallel(int n, F f) {
    if (n == 1) {
        f(0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve((size_t)n);
    for (int c = 0; c < n; c++) th.emplace_back(f, c);
    for (auto& t : th) t.join();
}

knn_status parse_all(const char* text, size_t len, const knn_spectra_opts* opts, knn_spectra** out) {
    if (!out) return fail(KNN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!text && len) return fail(KNN_EINVAL, "text is NULL");
    knn_spectra_opts o{};
    if (opts) o = *opts;
    if (o.mz_scale == 0.0) o.mz_scale = 10.0;
    if (!(o.mz_scale > 0.0) || !std::isfinite(o.mz_scale)) return fail(KNN_EINVAL, "mz_scale must be positive");
    if (!(o.min_intensity >= 0.0) || !std::isfinite(o.min_intensity))
        return fail(KNN_EINVAL, "min_intensity must be >= 0");
    if (o.dim < 0) return fail(KNN_EINVAL, "dim must be >= 0");
    if (o.merge != KNN_MERGE_MAX && o.merge != KNN_MERGE_SUM) return fail(KNN_EINVAL, "unknown merge rule");
    if (o.weights != KNN_SPECTRA_F32 && o.weights != KNN_SPECTRA_U8) return fail(KNN_EINVAL, "unknown weight type");
    if (o.chunk_bytes < 0) return fail(KNN_EINVAL, "chunk_bytes must be >= 0");
    knn_spectra_format fmt = o.format;
    if (fmt == KNN_SPECTRA_AUTO) {
        fmt = detect(text, len);
        if (fmt == KNN_SPECTRA_AUTO) return fail(KNN_EINVAL, "neither MGF nor MS2 (first line)");
    } else if (fmt != KNN_SPECTRA_MGF && fmt != KNN_SPECTRA_MS2) {
        return fail(KNN_EINVAL, "unknown format");
    }
    knn_spectra* sp = nullptr;
    try {
        // chunks of about chunk_bytes (4 MB), at most 4 per host thread and 256 in all
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const size_t chunk = o.chunk_bytes > 0 ? (size_t)o.chunk_bytes : ((size_t)4 << 20);
        const int T = (int)std::max<size_t>(1, std::min<size_t>({len / chunk, (size_t)hw * 4, 256}));
        const std::vector<size_t> cut = split_points(text, len, fmt, T);
        std::vector<int64_t> lines((size_t)T, 0);   // newlines in each chunk: line numbers of errors
        run_parallel(T, [&](int c) { lines[(size_t)c] = (int64_t)std::count(text + cut[c], text + cut[c + 1], '\n'); });
        std::vector<knn_spectra> parts((size_t)T);
        std::vector<knn_status> st((size_t)T, KNN_OK);
        std::vector<std::string> msg((size_t)T);
        std::vector<int64_t> max_d((size_t)T, -1);
        run_parallel(T, [&](int c) {
            try {
                Builder b(o, parts[(size_t)c]);
                Parser ps{text + cut[c], text + cut[c + 1]};
                for (int q = 0; q < c; q++) ps.line += lines[(size_t)q];
                st[(size_t)c] = fmt == KNN_SPECTRA_MS2 ? parse_ms2(ps, b) : parse_mgf(ps, b, c == T - 1);
                max_d[(size_t)c] = b.max_d;
                if (st[(size_t)c] != KNN_OK) msg[(size_t)c] = knn_last_error();   // this thread's message
            } catch (const std::bad_alloc&) {
                st[(size_t)c] = KNN_ENOMEM;
                msg[(size_t)c] = "host allocation failed while reading spectra";
            }
        });
        for (int c = 0; c < T; c++)   // the first error in file order
            if (st[(size_t)c] != KNN_OK) return fail(st[(size_t)c], "%s", msg[(size_t)c].c_str());
        sp = new knn_spectra();
        sp->dtype = o.weights == KNN_SPECTRA_U8 ? KNN_U8 : KNN_F32;
        size_t rows = 0, nnz = 0;
        for (const knn_spectra& q : parts) {
            rows += q.indptr.size() - 1;
            nnz += q.indices.size();
        }
        sp->indptr.reserve(rows + 1);
        sp->indices.reserve(nnz);
        if (sp->dtype == KNN_U8) sp->values_u8.reserve(nnz);
        else sp->values_f32.reserve(nnz);
        int64_t md = -1;
        for (int c = 0; c < T; c++) {
            knn_spectra& q = parts[(size_t)c];
            const int64_t base = (int64_t)sp->indices.size();
            for (size_t i = 1; i < q.indptr.size(); i++) sp->indptr.push_back(base + q.indptr[i]);
            sp->indices.insert(sp->indices.end(), q.indices.begin(), q.indices.end());
            sp->values_f32.insert(sp->values_f32.end(), q.values_f32.begin(), q.values_f32.end());
            sp->values_u8.insert(sp->values_u8.end(), q.values_u8.begin(), q.values_u8.end());
            sp->info.n_spectra += q.info.n_spectra;
            sp->info.n_peaks += q.info.n_peaks;
            sp->info.n_dropped += q.info.n_dropped;
            sp->info.n_merged += q.info.n_merged;
            md = std::max(md, max_d[(size_t)c]);
            q = knn_spectra();   // the part's memory goes back once it is copied
        }
        sp->dim = o.dim > 0 ? o.dim : (int32_t)std::max<int64_t>(1, md + 1);
        sp->info.n_features = (int64_t)sp->indices.size();
        sp->info.dim = sp->dim;
        sp->info.dtype = sp->dtype;
    } catch (const std::bad_alloc&) {
        delete sp;
        return fail(KNN_ENOMEM, "host allocation failed while reading spectra");
    } catch (const std::system_error& e) {   // a thread could not be started
        delete sp;
        return fail(KNN_ENOMEM, "reading spectra: %s", e.what());
    }
    *out = sp;
    return KNN_OK;
}

}  // namespace

extern "C" knn_status knn_spectra_parse(const char* text, size_t len, const knn_spectra_opts* opts,
                                        knn_spectra** out) {
    return parse_all(text, len, opts, out);
}

extern "C" knn_status knn_spectra_read(const char* path, const knn_spectra_opts* opts, knn_spectra** out) {
    if (!out) return fail(KNN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!path) return fail(KNN_EINVAL, "path is NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(KNN_EINVAL, "cannot open %s: %s", path, strerror(errno));
    std::string text;
    try {
        // one read into a buffer of the file's size, then whatever follows (a file that
        // grows meanwhile, or one whose size is not known up front)
        long size = -1;
        if (fseek(f, 0, SEEK_END) == 0) size = ftell(f);
        if (fseek(f, 0, SEEK_SET) != 0) size = -1;
        if (size > 0) {
            text.resize((size_t)size);
            text.resize(fread(&text[0], 1, (size_t)size, f));
        }
        char buf[1 << 16];
        size_t n;
        while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    } catch (const std::bad_alloc&) {
        fclose(f);
        return fail(KNN_ENOMEM, "host allocation failed while reading %s", path);
    }
    const bool bad = ferror(f) != 0;
    fclose(f);
    if (bad) return fail(KNN_EINVAL, "read error on %s", path);
    return parse_all(text.data(), text.size(), opts, out);
}

extern "C" knn_status knn_spectra_csr(const knn_spectra* sp, knn_csr* out) {
    if (!sp || !out) return fail(KNN_EINVAL, "NULL argument");
    out->n_rows = (int64_t)sp->indptr.size() - 1;
    out->dim = sp->dim;
    out->dtype = sp->dtype;
    out->indptr = sp->indptr.data();
    out->indices = sp->indices.data();
    out->values = sp->dtype == KNN_U8 ? (const void*)sp->values_u8.data() : (const void*)sp->values_f32.data();
    out->on_device = 0;
    return KNN_OK;
}

extern "C" knn_status knn_spectra_get_info(const knn_spectra* sp, knn_spectra_info* info) {
    if (!sp || !info) return fail(KNN_EINVAL, "NULL argument");
    *info = sp->info;
    return KNN_OK;
}

extern "C" void knn_spectra_free(knn_spectra* sp) { delete sp; }
