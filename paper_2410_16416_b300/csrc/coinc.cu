// Coincidence generator (the stage after the filter in Sec. II.A): pairs of
// triggers from two detectors found with the same template within the
// light-travel time.  Host code only; it runs on triggers already popped.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "lloid.h"

void set_last_error(const std::string &msg);

namespace {

// trigger indices ordered by (template, sample, index)
std::vector<int64_t> order_of(const sb_trigger *t, int64_t n) {
    std::vector<int64_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [t](int64_t x, int64_t y) {
        if (t[x].template_id != t[y].template_id) return t[x].template_id < t[y].template_id;
        if (t[x].sample != t[y].sample) return t[x].sample < t[y].sample;
        return x < y;
    });
    return idx;
}

}  // namespace

extern "C" int sb_coincidences(const sb_trigger *a, int64_t n_a, const sb_trigger *b, int64_t n_b,
                               int64_t max_dt_samples, sb_coinc *out, int64_t cap, int64_t *n_out) {
    if (!n_out || n_a < 0 || n_b < 0 || (n_a > 0 && !a) || (n_b > 0 && !b) || max_dt_samples < 0 || cap < 0 ||
        (cap > 0 && !out)) {
        set_last_error("sb_coincidences: bad argument");
        return SB_EINVAL;
    }
    const std::vector<int64_t> ia = order_of(a, n_a), ib = order_of(b, n_b);
    // sweep both lists template by template; for each A trigger, the B triggers of its template
    // within +-max_dt form a contiguous run, found from the previous A trigger's run start
    std::vector<sb_coinc> res;
    int64_t jb = 0;
    for (int64_t p = 0; p < n_a; ++p) {
        const sb_trigger &ta = a[ia[p]];
        while (jb < n_b && (b[ib[jb]].template_id < ta.template_id ||
                            (b[ib[jb]].template_id == ta.template_id && b[ib[jb]].sample < ta.sample - max_dt_samples)))
            ++jb;
        for (int64_t q = jb; q < n_b; ++q) {
            const sb_trigger &tb = b[ib[q]];
            if (tb.template_id != ta.template_id || tb.sample > ta.sample + max_dt_samples) break;
            sb_coinc c{};
            c.template_id = ta.template_id;
            c.index_a = ia[p];
            c.index_b = ib[q];
            c.sample_a = ta.sample;
            c.sample_b = tb.sample;
            c.snr_a = ta.snr;
            c.snr_b = tb.snr;
            c.network_snr = (float)std::sqrt((double)ta.snr * ta.snr + (double)tb.snr * tb.snr);
            res.push_back(c);
        }
    }
    // (template, sample_a, sample_b, index_a, index_b): the sweep gives (template, sample_a, index_a,
    // sample_b, index_b); equal sample_a with different index_a need the final sort
    std::sort(res.begin(), res.end(), [](const sb_coinc &x, const sb_coinc &y) {
        if (x.template_id != y.template_id) return x.template_id < y.template_id;
        if (x.sample_a != y.sample_a) return x.sample_a < y.sample_a;
        if (x.sample_b != y.sample_b) return x.sample_b < y.sample_b;
        if (x.index_a != y.index_a) return x.index_a < y.index_a;
        return x.index_b < y.index_b;
    });
    *n_out = (int64_t)res.size();
    const int64_t nw = std::min<int64_t>(cap, (int64_t)res.size());
    std::copy(res.begin(), res.begin() + nw, out);
    if ((int64_t)res.size() > cap) {
        set_last_error("sb_coincidences: " + std::to_string(res.size()) + " coincidences, room for " +
                       std::to_string(cap));
        return SB_EOVERFLOW;
    }
    return SB_OK;
}
