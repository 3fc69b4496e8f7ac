// ingest.cu — edge lists from files (Section II): the Graph Challenge's
// tab-separated files (one "u v [weight]" line per directed entry, 1-based
// ids) and Matrix Market coordinate files ("%%MatrixMarket matrix coordinate"
// header, a "rows cols entries" size line, then "i j [value]" 1-based).  Ids
// become 0-based; weights and values are ignored (any listed pair is an edge;
// cleaning is tc_build_csr's job).  Host code only: file reading is outside
// the timed path.
#include <cctype>
#include <cerrno>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tc_internal.cuh"

namespace {

struct Reader {
    FILE* f = nullptr;
    std::vector<char> line;
    int64_t lineno = 0;
    explicit Reader(const char* path) : f(std::fopen(path, "rb")), line(1 << 16) {}
    ~Reader() {
        if (f) std::fclose(f);
    }
    // next line (without its newline) or nullptr at the end; long lines grow the buffer
    const char* next() {
        size_t len = 0;
        for (;;) {
            if (!std::fgets(line.data() + len, (int)(line.size() - len), f)) {
                if (len == 0) return nullptr;
                break;
            }
            len += std::strlen(line.data() + len);
            if (len > 0 && line[len - 1] == '\n') break;
            if (len + 1 < line.size()) break;  // end of file without a newline
            line.resize(line.size() * 2);
        }
        while (len > 0 && (line[len - 1] == '\n' || line[len - 1] == '\r')) line[--len] = 0;
        ++lineno;
        return line.data();
    }
};

const char* skip_space(const char* p) {
    while (*p == ' ' || *p == '\t') ++p;
    return p;
}

// Parses one unsigned decimal id; false if there is none or it overflows.
bool parse_id(const char*& p, int64_t* out) {
    p = skip_space(p);
    if (*p < '0' || *p > '9') return false;
    int64_t v = 0;
    while (*p >= '0' && *p <= '9') {
        v = v * 10 + (*p - '0');
        if (v > (int64_t)INT32_MAX + 1) return false;
        ++p;
    }
    if (*p != 0 && *p != ' ' && *p != '\t') return false;
    *out = v;
    return true;
}

bool blank_or_comment(const char* p, bool mtx) {
    p = skip_space(p);
    return *p == 0 || *p == '%' || (!mtx && *p == '#');
}

int bad_line(const Reader& r, const char* what) {
    return tc::fail(TC_EINVAL, "tc_read_edges: line " + std::to_string(r.lineno) + ": " + what);
}

// One entry "u v [rest]" (1-based) -> 0-based pair.
int parse_pair(const Reader& r, const char* p, int64_t* u, int64_t* v) {
    if (!parse_id(p, u) || !parse_id(p, v)) return bad_line(r, "expected two vertex ids");
    if (*u < 1 || *v < 1 || *u > (int64_t)INT32_MAX || *v > (int64_t)INT32_MAX)
        return tc::fail(TC_ERANGE, "tc_read_edges: line " + std::to_string(r.lineno) +
                                       ": vertex id outside [1, 2^31 - 1]");
    *u -= 1;
    *v -= 1;
    return TC_OK;
}

int detect_format(const char* path) {
    const size_t n = std::strlen(path);
    auto ends = [&](const char* suf) {
        const size_t k = std::strlen(suf);
        return n >= k && std::strcmp(path + n - k, suf) == 0;
    };
    return ends(".mtx") || ends(".mm") ? 2 : 1;
}

}  // namespace

extern "C" int tc_read_edges(const char* path, int format, int32_t* src, int32_t* dst,
                             int64_t capacity, int64_t* m_out, int32_t* n_out) {
    if (!path || !m_out || !n_out) return tc::fail(TC_EINVAL, "tc_read_edges: NULL argument");
    if (format < 0 || format > 2) return tc::fail(TC_EINVAL, "tc_read_edges: unknown format");
    if ((src == nullptr) != (dst == nullptr))
        return tc::fail(TC_EINVAL, "tc_read_edges: src and dst must both be given or both NULL");
    const int fmt = format == 0 ? detect_format(path) : format;
    Reader r(path);
    if (!r.f)
        return tc::fail(TC_EINVAL, std::string("tc_read_edges: cannot open ") + path + ": " +
                                       std::strerror(errno));
    int64_t m = 0, max_id = -1, declared = -1, n_decl = 0;
    const char* p;
    if (fmt == 2) {
        p = r.next();
        if (!p || std::strncmp(p, "%%MatrixMarket", 14) != 0)
            return bad_line(r, "not a Matrix Market file");
        std::string h(p);
        for (auto& c : h) c = (char)std::tolower((unsigned char)c);
        if (h.find("matrix") == std::string::npos || h.find("coordinate") == std::string::npos)
            return bad_line(r, "only coordinate matrices hold edge lists");
        while ((p = r.next()) && blank_or_comment(p, true)) {
        }
        if (!p) return bad_line(r, "missing size line");
        int64_t rows = 0, cols = 0;
        if (!parse_id(p, &rows) || !parse_id(p, &cols) || !parse_id(p, &declared))
            return bad_line(r, "expected 'rows cols entries'");
        if (rows > (int64_t)INT32_MAX || cols > (int64_t)INT32_MAX)
            return tc::fail(TC_ERANGE, "tc_read_edges: matrix larger than 2^31 - 1 vertices");
        n_decl = rows > cols ? rows : cols;
    }
    while ((p = r.next())) {
        if (blank_or_comment(p, fmt == 2)) continue;
        int64_t u, v;
        if (int rc = parse_pair(r, p, &u, &v)) return rc;
        if (fmt == 2 && (u >= n_decl || v >= n_decl))
            return tc::fail(TC_ERANGE, "tc_read_edges: line " + std::to_string(r.lineno) +
                                           ": entry outside the declared size");
        if (src && m < capacity) {
            src[m] = (int32_t)u;
            dst[m] = (int32_t)v;
        }
        ++m;
        if (u > max_id) max_id = u;
        if (v > max_id) max_id = v;
    }
    if (std::ferror(r.f)) return tc::fail(TC_EINVAL, "tc_read_edges: read error");
    if (fmt == 2 && m != declared)
        return tc::fail(TC_EINVAL, "tc_read_edges: " + std::to_string(m) + " entries, " +
                                       std::to_string(declared) + " declared");
    *m_out = m;
    *n_out = (int32_t)(fmt == 2 ? n_decl : max_id + 1);
    if (src && m > capacity)
        return tc::fail(TC_EINVAL, "tc_read_edges: " + std::to_string(m) +
                                       " entries do not fit the capacity given");
    return TC_OK;
}
