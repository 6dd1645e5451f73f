// launch_shape.cu -- host-side choice of the z-chunk (planes per CTA) of a
// single-grid step launch.
//
// A launch is (tiles) xy tiles x (chunks) z-chunks of CTAs; each CTA marches
// its chunk plus one halo plane on each side.  The choice trades the halo
// planes that short chunks re-read against the imbalance of the last round of
// CTAs on the device's resident slots (SMs x CTAs per SM of that kernel):
//
// - Many rounds (16-plane chunks would fill four or more rounds of the
//   slots): chunks of 16 planes or more, about `target` CTAs (six rounds of
//   the kernel family's design occupancy).  A 512^3 sweep placed the optimum
//   there, and with many rounds the last one's imbalance is a small part of
//   the launch.
// - Few rounds: every chunk length from 4 to 64 planes is scored by the
//   makespan of a greedy dispatch of the CTAs, in launch order, to the slots:
//   a CTA takes (its planes + 1) units, and one that has to wait for a slot
//   2 units more (the next step's CTAs, launched early, compete for the slots
//   that free up).  The shortest makespan wins, ties to the longer chunk.
//   The launch order puts the short last chunk of each column last.  Fitted
//   to sweeps of 4 ... 48 planes (FP32, 96^3 ... 384^3, contact and periodic
//   faces, CF / TI / TI_n / stochastic rounding, 19 configurations): the
//   choice ran 1.5 % above the best measured one on average, 10 % at worst,
//   where chunks of 16 planes or more lost up to 2x on grids of 96^3 ... 192^3.
//   The model takes a CTA's speed as independent of the CTAs beside it on its
//   SM, which holds for the streaming kernels at three or four CTAs per SM;
//   kernels with fewer (TI_n: two, bound by instruction issue, where a CTA
//   left alone on an SM runs faster) keep the rule of many rounds.
#include <map>
#include <mutex>
#include <queue>
#include <tuple>
#include <vector>

#include "spfm_internal.h"

namespace spfm {

// makespan, in plane units, of `tiles` x ceil(nz / zc) CTAs dispatched in
// launch order to `slots` slots by a greedy scheduler (see above)
static long long dispatch_makespan(int tiles, int nz, int zc, int slots)
{
    constexpr long long h = 1, w = 2;
    const int chunks = (nz + zc - 1) / zc;
    const int last = nz - (chunks - 1) * zc;
    const long long d = zc + h, ds = last + h;
    const long long nfull = (long long)tiles * (last < zc ? chunks - 1 : chunks);
    const long long nshort = last < zc ? tiles : 0;
    // the equal CTAs first: r slots carry q + 1 of them, the others q, each
    // after the first on its slot having waited
    const long long q = nfull / slots, r = nfull % slots;
    auto load = [&](long long k) { return k == 0 ? 0 : k * d + (k - 1) * w; };
    long long span = load(q + (r > 0));
    if (nshort == 0) return span;
    // the short CTAs go to the slots that free first
    std::priority_queue<long long, std::vector<long long>, std::greater<long long>> free_at;
    for (long long i = 0; i < slots; ++i) free_at.push(load(i < r ? q + 1 : q));
    for (long long i = 0; i < nshort; ++i) {
        const long long t = free_at.top() + (nfull + i >= slots ? w : 0) + ds;
        free_at.pop();
        free_at.push(t);
        if (t > span) span = t;
    }
    return span;
}

static int model_zchunk(int tiles, int nz, int per_sm, int slots, int target)
{
    if (nz <= 4) return nz;
    const long long rounds16 = (long long)tiles * ((nz + 15) / 16);
    if (rounds16 >= 4LL * slots || per_sm < 3) {
        int chunks = (target + tiles - 1) / tiles;
        const int max_chunks = nz / 16 > 1 ? nz / 16 : 1;
        if (chunks > max_chunks) chunks = max_chunks;
        if (chunks < 1) chunks = 1;
        return (nz + chunks - 1) / chunks;
    }
    int best = 4;
    long long best_span = -1;
    const int hi = nz < 64 ? nz : 64;
    for (int zc = 4; zc <= hi; ++zc) {
        const long long span = dispatch_makespan(tiles, nz, zc, slots);
        if (best_span < 0 || span <= best_span) {
            best_span = span;
            best = zc;
        }
    }
    return best;
}

namespace {
std::mutex g_mu;
// (kernel, threads, device) -> resident CTAs per SM; (tiles, nz, slots, target) -> z-chunk
std::map<std::tuple<const void *, int, int>, int> g_occ;
std::map<std::tuple<int, int, int, int>, int> g_zc;
}  // namespace

int pick_zchunk(const void *kern, int threads, int tiles, int nz, int target)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::lock_guard<std::mutex> lock(g_mu);
    const auto ok = std::make_tuple(kern, threads, dev);
    auto o = g_occ.find(ok);
    int per_sm;
    if (o != g_occ.end()) {
        per_sm = o->second;
    } else {
        per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();   // the launch itself reports a kernel that cannot run
            per_sm = 1;
        }
        g_occ[ok] = per_sm;
    }
    const int slots = per_sm * sms;
    const auto zk = std::make_tuple(tiles, nz, slots, target);
    auto z = g_zc.find(zk);
    if (z != g_zc.end()) return z->second;
    if (g_zc.size() >= 4096) g_zc.clear();   // many grid shapes (a serving process): start over
    const int zc = model_zchunk(tiles, nz, per_sm, slots, target);
    g_zc[zk] = zc;
    return zc;
}

}  // namespace spfm

extern "C" int spfm_debug_pick_zchunk(int tiles, int nz, int per_sm, int sms, int target)
{
    if (tiles < 1 || nz < 1 || per_sm < 1 || sms < 1 || target < 1) return -1;
    return spfm::model_zchunk(tiles, nz, per_sm, per_sm * sms, target);
}
