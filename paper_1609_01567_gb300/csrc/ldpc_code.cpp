// Code tables: COO of H -> edge ids, CSC by variable, CSR by check, the edge
// permutation between the two orders, and check degree bins (host side), plus
// their upload to the device. Also the error-text plumbing of the C ABI.
//
// The edge numbering follows Section III-B: edge ids e are the COO entries
// stably sorted by variable (Table 1: e, v, c with segment start s, degree t
// and rank u); the check order is e stably sorted by check (Table 2: ebar,
// vbar, cbar, sbar, tbar, ubar).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ldpc_internal.h"

namespace ldpc {

static thread_local std::string g_last_error;

int set_error(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_error(cudaError_t e, const char *what) {
    return set_error(e == cudaErrorMemoryAllocation ? LDPC_ENOMEM : LDPC_ECUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

}  // namespace ldpc

using namespace ldpc;

static void free_device_tables(ldpc_code *c) {
    if (c->device < 0) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaFree(c->d.row_ptr);
    cudaFree(c->d.col_idx);
    cudaFree(c->d.col_ptr);
    cudaFree(c->d.edge_slot);
    cudaFree(c->d.bin_checks);
    cudaFree(c->d.bin_desc);
    cudaFree(c->d.phi_table);
    cudaFree(c->d.ms_table);
    cudaFree(c->d.wide_vars);
    cudaFree(c->enc_R);
    cudaFree(c->enc_colmap);
    c->enc_R = nullptr;
    c->enc_colmap = nullptr;
    free_host_stream(c);
    free_decode_graphs(c);
    free_workspace(c->ws);
    for (auto &p : c->prof) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    c->d = DeviceTables{};
    c->ws = Workspace{};
    if (prev >= 0) cudaSetDevice(prev);
}

// Chords of the tabulated phi: bucket key k spans [e_k, e_(k+1)), e_k the
// float with bits k << 17; on it phi(x) ~ a + b x through (e_k, phi(e_k)) and
// (e_(k+1), phi(e_(k+1))), computed in double and stored as float.
static std::vector<float2> phi_chords() {
    auto edge = [](uint32_t key) {
        uint32_t bits = key << 17;
        float f;
        memcpy(&f, &bits, sizeof f);
        return (double)f;
    };
    auto phi = [](double x) { return std::log1p(2.0 / std::expm1(x)); };
    std::vector<float2> t((size_t)kPhiTableSize);
    for (int i = 0; i < kPhiTableSize; ++i) {
        const double lo = edge(kPhiKey0 + (uint32_t)i), hi = edge(kPhiKey0 + (uint32_t)i + 1);
        const double plo = phi(lo), phi_hi = phi(hi);
        const double b = (phi_hi - plo) / (hi - lo);
        t[(size_t)i] = make_float2((float)(plo - b * lo), (float)b);
    }
    return t;
}

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
    size_t bytes = sizeof(T) * (src.empty() ? 1 : src.size());
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

extern "C" int ldpc_code_create(int32_t m, int32_t n, int64_t nnz, const int32_t *rows, const int32_t *cols,
                                const ldpc_code_opts_t *opts, ldpc_code_t **out) {
    if (!out) return set_error(LDPC_EINVAL, "ldpc_code_create: out is NULL");
    *out = nullptr;
    if (m < 0 || n < 0) return set_error(LDPC_EINVAL, "ldpc_code_create: negative size m=%d n=%d", m, n);
    if (nnz < 0 || nnz > INT32_MAX)
        return set_error(LDPC_EINVAL, "ldpc_code_create: nnz=%lld outside [0, 2^31-1]", (long long)nnz);
    if (nnz > 0 && (!rows || !cols)) return set_error(LDPC_EINVAL, "ldpc_code_create: rows/cols is NULL");
    int device = opts ? opts->device : 0;

    ldpc_code *c = new (std::nothrow) ldpc_code();
    if (!c) return set_error(LDPC_ENOMEM, "ldpc_code_create: out of host memory");
    try {
        c->m = m;
        c->n = n;
        c->E = nnz;
        const int64_t E = nnz;
        for (int64_t t = 0; t < E; ++t) {
            if (rows[t] < 0 || rows[t] >= m || cols[t] < 0 || cols[t] >= n) {
                delete c;
                return set_error(LDPC_EINVAL, "ldpc_code_create: entry %lld = (%d, %d) outside H (%d x %d)",
                                 (long long)t, rows[t], cols[t], m, n);
            }
        }
        // CSC by variable; edge ids = stable sort of the COO by column.
        c->col_ptr.assign((size_t)n + 1, 0);
        for (int64_t t = 0; t < E; ++t) c->col_ptr[cols[t] + 1]++;
        for (int32_t j = 0; j < n; ++j) c->col_ptr[j + 1] += c->col_ptr[j];
        c->var_of_edge.resize(E);
        c->chk_of_edge.resize(E);
        {
            std::vector<int32_t> fill(c->col_ptr.begin(), c->col_ptr.end() - 1);
            for (int64_t t = 0; t < E; ++t) {
                int32_t e = fill[cols[t]]++;
                c->var_of_edge[e] = cols[t];
                c->chk_of_edge[e] = rows[t];
            }
        }
        // repeated (row, column): within one column, every check at most once
        {
            std::vector<int32_t> seen((size_t)m, -1);
            for (int32_t j = 0; j < n; ++j) {
                for (int32_t e = c->col_ptr[j]; e < c->col_ptr[j + 1]; ++e) {
                    int32_t i = c->chk_of_edge[e];
                    if (seen[i] == j) {
                        delete c;
                        return set_error(LDPC_EDUP, "ldpc_code_create: H[%d][%d] appears more than once", i, j);
                    }
                    seen[i] = j;
                }
            }
        }
        // CSR by check; check order = stable sort of edge ids by check.
        c->row_ptr.assign((size_t)m + 1, 0);
        for (int64_t e = 0; e < E; ++e) c->row_ptr[c->chk_of_edge[e] + 1]++;
        for (int32_t i = 0; i < m; ++i) c->row_ptr[i + 1] += c->row_ptr[i];
        c->edge_of_slot.resize(E);
        c->col_idx.resize(E);
        c->edge_slot.resize(E);
        {
            std::vector<int32_t> fill(c->row_ptr.begin(), c->row_ptr.end() - 1);
            for (int64_t e = 0; e < E; ++e) {
                int32_t k = fill[c->chk_of_edge[e]]++;
                c->edge_of_slot[k] = (int32_t)e;
                c->col_idx[k] = c->var_of_edge[e];
                c->edge_slot[e] = k;
            }
        }
        for (int32_t i = 0; i < m; ++i) c->max_cdeg = std::max(c->max_cdeg, c->row_ptr[i + 1] - c->row_ptr[i]);
        for (int32_t j = 0; j < n; ++j) {
            c->max_vdeg = std::max(c->max_vdeg, c->col_ptr[j + 1] - c->col_ptr[j]);
            if (c->col_ptr[j + 1] - c->col_ptr[j] > kWideVarDegree) c->wide_vars.push_back(j);
        }
        // IRA form: column k + i joins checks i and i + 1 (the last one only
        // check m - 1), k = n - m
        if (n >= m) {
            const int32_t k = n - m;
            bool stair = true;
            for (int32_t i = 0; i < m && stair; ++i) {
                const int32_t j = k + i, d = c->col_ptr[j + 1] - c->col_ptr[j];
                const int32_t e = c->col_ptr[j];
                if (i + 1 < m)
                    stair = d == 2 && std::min(c->chk_of_edge[e], c->chk_of_edge[e + 1]) == i &&
                            std::max(c->chk_of_edge[e], c->chk_of_edge[e + 1]) == i + 1;
                else
                    stair = d == 1 && c->chk_of_edge[e] == i;
            }
            if (stair) c->ira_k = k;
        }
        // check degree bins (degree-0 checks carry no message and are skipped)
        for (int b = 0; b < kNumCheckBins; ++b) {
            c->bin_off[b] = (int32_t)c->bin_checks.size();
            int lo = b == 0 ? 1 : kBinMaxDegree[b - 1] + 1;
            int hi = kBinMaxDegree[b];
            for (int32_t i = 0; i < m; ++i) {
                int d = c->row_ptr[i + 1] - c->row_ptr[i];
                if (d >= lo && d <= hi) {
                    c->bin_checks.push_back(i);
                    c->bin_max_degree[b] = std::max(c->bin_max_degree[b], d);
                }
            }
        }
        c->bin_off[kNumCheckBins] = (int32_t)c->bin_checks.size();
        c->bin_desc.reserve(c->bin_checks.size());
        for (int32_t i : c->bin_checks) c->bin_desc.push_back(make_int2(c->row_ptr[i], c->row_ptr[i + 1] - c->row_ptr[i]));
    } catch (const std::bad_alloc &) {
        delete c;
        return set_error(LDPC_ENOMEM, "ldpc_code_create: out of host memory");
    }

    if (device >= 0) {
        int count = 0;
        cudaError_t e = cudaGetDeviceCount(&count);
        if (e != cudaSuccess || device >= count) {
            delete c;
            if (e != cudaSuccess) return cuda_error(e, "ldpc_code_create: cudaGetDeviceCount");
            return set_error(LDPC_EINVAL, "ldpc_code_create: device %d not present (%d devices)", device, count);
        }
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        c->device = device;
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
        if ((e = upload(&c->d.row_ptr, c->row_ptr)) != cudaSuccess ||
            (e = upload(&c->d.col_idx, c->col_idx)) != cudaSuccess ||
            (e = upload(&c->d.col_ptr, c->col_ptr)) != cudaSuccess ||
            (e = upload(&c->d.edge_slot, c->edge_slot)) != cudaSuccess ||
            (e = upload(&c->d.bin_checks, c->bin_checks)) != cudaSuccess ||
            (e = upload(&c->d.bin_desc, c->bin_desc)) != cudaSuccess ||
            (e = upload(&c->d.phi_table, phi_chords())) != cudaSuccess ||
            (e = upload(&c->d.wide_vars, c->wide_vars)) != cudaSuccess ||
            (e = upload(&c->d.ms_table, std::vector<float2>((size_t)c->max_cdeg + 1, make_float2(1.0f, 0.0f)))) !=
                cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->ws.last_use, cudaEventDisableTiming)) != cudaSuccess) {
            int st = cuda_error(e, "ldpc_code_create: device upload");
            free_device_tables(c);
            delete c;
            if (prev >= 0) cudaSetDevice(prev);
            return st;
        }
        if (prev >= 0) cudaSetDevice(prev);
    }
    *out = c;
    return LDPC_OK;
}

extern "C" int ldpc_code_create_qc(int32_t mb, int32_t nb, int32_t Z, int64_t n_entries, const int32_t *brow,
                                   const int32_t *bcol, const int32_t *shift, const ldpc_code_opts_t *opts,
                                   ldpc_code_t **out) {
    if (!out) return set_error(LDPC_EINVAL, "ldpc_code_create_qc: out is NULL");
    *out = nullptr;
    if (mb < 0 || nb < 0 || Z < 1 || n_entries < 0)
        return set_error(LDPC_EINVAL, "ldpc_code_create_qc: bad size mb=%d nb=%d Z=%d entries=%lld", mb, nb, Z,
                         (long long)n_entries);
    if ((int64_t)mb * Z > INT32_MAX || (int64_t)nb * Z > INT32_MAX || n_entries * Z > INT32_MAX)
        return set_error(LDPC_EINVAL, "ldpc_code_create_qc: lifted code exceeds 2^31-1 rows, columns or edges");
    if (n_entries > 0 && (!brow || !bcol || !shift)) return set_error(LDPC_EINVAL, "ldpc_code_create_qc: NULL entry array");
    std::vector<int32_t> rows, cols;
    try {
        rows.resize((size_t)(n_entries * Z));
        cols.resize((size_t)(n_entries * Z));
    } catch (const std::bad_alloc &) {
        return set_error(LDPC_ENOMEM, "ldpc_code_create_qc: out of host memory");
    }
    for (int64_t b = 0; b < n_entries; ++b) {
        if (brow[b] < 0 || brow[b] >= mb || bcol[b] < 0 || bcol[b] >= nb || shift[b] < 0 || shift[b] >= Z)
            return set_error(LDPC_EINVAL, "ldpc_code_create_qc: entry %lld = (%d, %d, shift %d) outside %d x %d, Z %d",
                             (long long)b, brow[b], bcol[b], shift[b], mb, nb, Z);
        // circulant P^s: row t of the block joins column (t + s) mod Z
        for (int32_t t = 0; t < Z; ++t) {
            const size_t o = (size_t)b * Z + t;
            rows[o] = brow[b] * Z + t;
            cols[o] = bcol[b] * Z + (int32_t)(((int64_t)t + shift[b]) % Z);
        }
    }
    int st = ldpc_code_create(mb * Z, nb * Z, n_entries * Z, rows.data(), cols.data(), opts, out);
    if (st == LDPC_EDUP) set_error(LDPC_EDUP, "ldpc_code_create_qc: a base entry repeats (same block, same shift)");
    return st;
}

extern "C" void ldpc_code_destroy(ldpc_code_t *code) {
    if (!code) return;
    free_device_tables(code);
    delete code;
}

extern "C" int ldpc_code_set_rule_table(ldpc_code_t *c, int32_t n_degrees, const float *alpha_by_degree,
                                        const float *beta_by_degree) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_code_set_rule_table: code is NULL");
    if (n_degrees < 1 || !alpha_by_degree)
        return set_error(LDPC_EINVAL, "ldpc_code_set_rule_table: need n_degrees >= 1 and alpha_by_degree");
    for (int32_t t = 0; t < n_degrees; ++t) {
        const float a = alpha_by_degree[t], b = beta_by_degree ? beta_by_degree[t] : 0.0f;
        if (!(a > 0.0f) || !std::isfinite(a) || !(b >= 0.0f) || !std::isfinite(b))
            return set_error(LDPC_EINVAL, "ldpc_code_set_rule_table: entry %d = (%g, %g) needs alpha > 0, beta >= 0",
                             t, (double)a, (double)b);
    }
    if (c->device < 0) return set_error(LDPC_EINVAL, "ldpc_code_set_rule_table: host-only code");
    // one entry per degree 0 .. max check degree; degrees past the caller's
    // table take its last entry
    std::vector<float2> tab((size_t)c->max_cdeg + 1);
    for (size_t d = 0; d < tab.size(); ++d) {
        const int32_t t = (int64_t)d < n_degrees ? (int32_t)d : n_degrees - 1;
        tab[d] = make_float2(alpha_by_degree[t], beta_by_degree ? beta_by_degree[t] : 0.0f);
    }
    std::lock_guard<std::mutex> lock(c->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpy(c->d.ms_table, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_code_set_rule_table: cudaMemcpy");
    c->ms_table_set = true;
    return LDPC_OK;
}

extern "C" int ldpc_code_info(const ldpc_code_t *c, ldpc_code_info_t *info) {
    if (!c || !info) return set_error(LDPC_EINVAL, "ldpc_code_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->m = c->m;
    info->n = c->n;
    info->n_edges = c->E;
    info->max_check_degree = c->max_cdeg;
    info->max_var_degree = c->max_vdeg;
    info->mean_check_degree = c->m ? (double)c->E / c->m : 0.0;
    info->mean_var_degree = c->n ? (double)c->E / c->n : 0.0;
    info->n_check_bins = kNumCheckBins;
    for (int b = 0; b < kNumCheckBins; ++b) {
        info->check_bin_max_degree[b] = kBinMaxDegree[b];
        info->check_bin_count[b] = c->bin_off[b + 1] - c->bin_off[b];
    }
    info->device = c->device;
    info->ira_k = c->ira_k;
    return LDPC_OK;
}

extern "C" int ldpc_code_tables(const ldpc_code_t *c, int32_t *v, int32_t *cc, int32_t *t, int32_t *s, int32_t *u,
                                int32_t *ebar, int32_t *vbar, int32_t *cbar, int32_t *tbar, int32_t *sbar,
                                int32_t *ubar) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_code_tables: code is NULL");
    for (int64_t e = 0; e < c->E; ++e) {
        int32_t j = c->var_of_edge[e];
        if (v) v[e] = j;
        if (cc) cc[e] = c->chk_of_edge[e];
        if (t) t[e] = c->col_ptr[j + 1] - c->col_ptr[j];
        if (s) s[e] = c->col_ptr[j];
        if (u) u[e] = (int32_t)e - c->col_ptr[j];
    }
    for (int32_t i = 0; i < c->m; ++i) {
        for (int32_t k = c->row_ptr[i]; k < c->row_ptr[i + 1]; ++k) {
            if (ebar) ebar[k] = c->edge_of_slot[k];
            if (vbar) vbar[k] = c->col_idx[k];
            if (cbar) cbar[k] = i;
            if (tbar) tbar[k] = c->row_ptr[i + 1] - c->row_ptr[i];
            if (sbar) sbar[k] = c->row_ptr[i];
            if (ubar) ubar[k] = k - c->row_ptr[i];
        }
    }
    return LDPC_OK;
}

extern "C" const char *ldpc_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *ldpc_version(void) { return "ldpc-gb300 0.1 (sm_103a)"; }
