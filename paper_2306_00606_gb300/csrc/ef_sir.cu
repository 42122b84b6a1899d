// SIR epidemic simulation of libef (Section 3.1's model; Section 3.2's
// measurements: final size, global outbreaks, epidemic length, time to
// peak, and the spreading power of order k from the infection tree).
//
// Discrete time, synchronous steps t = 0, 1, ... on the states at the start
// of the step:
//   - every node u infected at the start of step t tries once each neighbour
//     x susceptible at that time, with success when the draw
//     R(sim, t, u, x) < floor(beta 2^32); x becomes infected at the end of
//     the step when any try succeeds, its infector being the smallest such u;
//   - u recovers at the end of step t when R(sim, t, u, 2^32 - 1) <
//     floor(gamma 2^32);
//   - the epidemic ends at the first t with no infected node (its length).
// R is Philox4x32-10 (Salmon et al., SC 2011) with counter (sim, t, u, x)
// and key = the 64-bit seed, first output word: a simulation's course
// depends on its id and the seed only, not on the batch or the launch.
//
// Layout: per (simulation s, node v): a susceptibility bit (bit v & 31 of
// word s * W + v / 32, W = ceil(n / 32): the only state the tries read, 1/8
// of a state byte so that it stays in L2), at s * n + v the infector
// (parent) and the smallest successful infector of the current step (cand).
// Infected and recovered nodes are the ones without the bit and with a
// parent, immune nodes the ones without either; recovery only leaves the
// frontier.  The infected (s, u) pairs of a step form a frontier list of
// 64-bit entries s << 32 | u; a step appends survivors and new infections
// to the other list.  Kernels of a step:
//   k_sir_spread  4 frontier entries per warp, 8 lanes each over the
//                 entry's neighbours: tries, cand by atomicMin (the first
//                 success appends x), the recovery draw (survivors append);
//                 entries of degree > SIR_HEAVY are listed for
//   k_sir_spread_heavy  a CTA per listed entry over its neighbours (hubs
//                 would otherwise hold a warp for hundreds of rounds)
//   k_sir_commit  over the new list: a node still susceptible becomes
//                 infected with parent = cand
//   k_sir_stats   per simulation: peak, peak step, length; clears the
//                 emptied list's count for the next step
// Launch shapes read the list counts from device memory, so the host only
// reads the number of active simulations every SIR_CHECK steps.
#include "ef_internal.cuh"

namespace ef {

constexpr int32_t NO_CAND = 0x7fffffff;
constexpr uint32_t RECOVER_WORD = 0xffffffffu;
constexpr int SIR_HEAVY = 64;   // frontier entries of higher degree are tried by a CTA each

// Philox4x32-10, first output word only.
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key) {
    uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}

__device__ __forceinline__ uint64_t sir_entry(int s, int v) { return (uint64_t)(uint32_t)s << 32 | (uint32_t)v; }

__device__ __forceinline__ int64_t sir_words(int32_t n) { return ((int64_t)n + 31) >> 5; }

__device__ __forceinline__ bool susceptible(const uint32_t *susc, int64_t wrow, int x) {
    return (__ldg(susc + wrow + (x >> 5)) >> (x & 31)) & 1u;
}

// Susceptibility words (all nodes but the immune ones), parents and
// candidates of every (simulation, node).
__global__ void k_sir_init(int32_t B, int32_t n, const uint8_t *__restrict__ immune, int32_t num_sets,
                           const int32_t *__restrict__ imm_set, SirState st) {
    const int64_t W = sir_words(n), words = (int64_t)B * W, total = (int64_t)B * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
        const int s = (int)(i / W);
        const int v0 = (int)(i - (int64_t)s * W) * 32;
        uint32_t w = 0;
        int set = -1;
        if (imm_set) {
            set = imm_set[s];
            if (set >= num_sets) {
                atomicOr(st.err, ERRB_SIR_ARG);
                set = -1;
            }
        }
        for (int b = 0; b < 32 && v0 + b < n; ++b)
            if (set < 0 || !immune[(int64_t)set * n + v0 + b]) w |= 1u << b;
        st.susc[i] = w;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        st.parent[i] = -1;
        st.cand[i] = NO_CAND;
    }
}

// The index cases and the first frontier (an immune index case is an error).
__global__ void k_sir_seed(const int32_t *__restrict__ index_cases, int32_t B, int32_t n, SirState st) {
    const int64_t W = sir_words(n);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < B; s += gridDim.x * blockDim.x) {
        const int u = index_cases[s];
        st.peak[s] = 1;
        st.peak_step[s] = 0;
        st.length[s] = 0;
        st.count[s] = 0;
        st.done[s] = 0;
        st.fsize[s] = 1;
        if (u < 0 || u >= n || !susceptible(st.susc, s * W, u)) {
            atomicOr(st.err, ERRB_SIR_ARG);
            st.done[s] = 1;   // no frontier entry: the simulation does not run
            st.fsize[s] = 0;
            continue;
        }
        st.susc[s * W + (u >> 5)] &= ~(1u << (u & 31));   // one index case per row of words
        st.parent[(int64_t)s * n + u] = u;
        st.list[0][s] = sir_entry(s, u);
    }
}

__device__ __forceinline__ void sir_append(bool app, uint64_t ent, uint64_t *__restrict__ nxt,
                                           int64_t *__restrict__ cnxt, int32_t *__restrict__ count);

// One step over the frontier list `cur` (count *ccur), appending to `nxt`;
// entries of degree > SIR_HEAVY go to the heavy list instead.
__global__ void __launch_bounds__(256) k_sir_spread(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                    int32_t n, int32_t t, SirStep p, SirState st,
                                                    const uint64_t *__restrict__ cur, const int64_t *__restrict__ ccur,
                                                    uint64_t *__restrict__ nxt, int64_t *__restrict__ cnxt) {
    const int lane = threadIdx.x & 31, oct = lane >> 3, l8 = lane & 7;
    const int64_t total = *ccur;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4; base < total;
         base += nwarps * 4) {
        const int64_t item = base + oct;
        const bool valid = item < total;
        int s = 0, u = 0, a = 0, D = 0;
        if (valid) {
            const uint64_t e = cur[item];
            s = (int)(e >> 32);
            u = (int)(uint32_t)e;
            a = rp[u];
            D = rp[u + 1] - a;
            if (D > SIR_HEAVY) {
                // tried by k_sir_spread_heavy, a CTA per entry
                if (l8 == 0) st.heavy[atomicAdd((unsigned long long *)st.heavy_count, 1ull)] = e;
                D = 0;
            }
        }
        const uint32_t sim = (uint32_t)(p.sim_base + s);
        const int64_t row = (int64_t)s * n, wrow = s * sir_words(n);
        // recovery (lane 0 of the octet): survivors stay in the frontier
        bool app = false;
        uint64_t ent = 0;
        if (valid && l8 == 0) {
            const uint32_t w = philox_w0(sim, (uint32_t)t, (uint32_t)u, RECOVER_WORD, p.seed);
            if ((uint64_t)w >= p.gamma_thr) {
                app = true;
                ent = sir_entry(s, u);
            }
        }
        int kmax = D;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
        for (int k0 = 0;; k0 += 8) {
            sir_append(app, ent, nxt, cnxt, st.count);   // this round's entries
            if (k0 >= kmax) break;
            app = false;
            const int k = k0 + l8;
            if (valid && k < D) {
                const int x = ci[a + k];
                if (susceptible(st.susc, wrow, x)) {
                    const uint32_t w = philox_w0(sim, (uint32_t)t, (uint32_t)u, (uint32_t)x, p.seed);
                    if ((uint64_t)w < p.beta_thr) {
                        const int old = atomicMin(st.cand + row + x, u);
                        if (old == NO_CAND) {
                            app = true;
                            ent = sir_entry(s, x);
                        }
                    }
                }
            }
        }
    }
}

// Appends the lanes' entries (app) to nxt with one list atomic per warp and
// one count update per simulation; every lane of the warp calls it.
__device__ __forceinline__ void sir_append(bool app, uint64_t ent, uint64_t *__restrict__ nxt,
                                           int64_t *__restrict__ cnxt, int32_t *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(FULL, app);
    if (!bal) return;
    int64_t pos = 0;
    const int leader = __ffs(bal) - 1;
    if (lane == leader) pos = atomicAdd((unsigned long long *)cnxt, (unsigned long long)__popc(bal));
    pos = __shfl_sync(FULL, pos, leader);
    if (app) {
        nxt[pos + __popc(bal & ((1u << lane) - 1u))] = ent;
        const int es = (int)(ent >> 32);
        const unsigned peers = __match_any_sync(bal, es);
        if (lane == __ffs(peers) - 1) atomicAdd(count + es, __popc(peers));
    }
}

// The tries of the frontier entries of degree > SIR_HEAVY: a CTA per entry,
// its threads over the neighbours.
__global__ void __launch_bounds__(256) k_sir_spread_heavy(const int32_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci, int32_t n, int32_t t,
                                                          SirStep p, SirState st, uint64_t *__restrict__ nxt,
                                                          int64_t *__restrict__ cnxt) {
    const int64_t total = *st.heavy_count;
    for (int64_t h = blockIdx.x; h < total; h += gridDim.x) {
        const uint64_t e = st.heavy[h];
        const int s = (int)(e >> 32), u = (int)(uint32_t)e;
        const int a = rp[u], D = rp[u + 1] - a;
        const uint32_t sim = (uint32_t)(p.sim_base + s);
        const int64_t row = (int64_t)s * n, wrow = s * sir_words(n);
        for (int k0 = 0; k0 < D; k0 += blockDim.x) {
            const int k = k0 + threadIdx.x;
            bool app = false;
            uint64_t ent = 0;
            if (k < D) {
                const int x = ci[a + k];
                if (susceptible(st.susc, wrow, x)) {
                    const uint32_t w = philox_w0(sim, (uint32_t)t, (uint32_t)u, (uint32_t)x, p.seed);
                    if ((uint64_t)w < p.beta_thr && atomicMin(st.cand + row + x, u) == NO_CAND) {
                        app = true;
                        ent = sir_entry(s, x);
                    }
                }
            }
            sir_append(app, ent, nxt, cnxt, st.count);
        }
    }
}

// New infections of the step: the entries of `nxt` whose node is still
// susceptible (the others are survivors).  Each entry is listed once, so its
// bit is read plainly and cleared atomically (its word is shared).
__global__ void k_sir_commit(int32_t n, SirState st, const uint64_t *__restrict__ nxt,
                             const int64_t *__restrict__ cnxt) {
    const int64_t total = *cnxt, W = sir_words(n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = nxt[i];
        const int s = (int)(e >> 32), x = (int)(uint32_t)e;
        const int64_t j = (int64_t)s * n + x;
        uint32_t *word = st.susc + s * W + (x >> 5);
        const uint32_t bit = 1u << (x & 31);
        if (*word & bit) {
            atomicAnd(word, ~bit);
            st.parent[j] = st.cand[j];
            st.cand[j] = NO_CAND;
            atomicAdd(st.fsize + s, 1);
        }
    }
}

// After step t: |I_{t+1}| per simulation is count[s].  active[t & 1] counts
// warps with a simulation still running; active[(t + 1) & 1] is cleared for
// the next step.
__global__ void k_sir_stats(int32_t B, int32_t t, SirState st, int64_t *__restrict__ ccur,
                            int64_t *__restrict__ active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *ccur = 0;   // the list just read is the next step's output
        *st.heavy_count = 0;
        active[(t + 1) & 1] = 0;
    }
    int act = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < B; s += gridDim.x * blockDim.x) {
        const int c = st.count[s];
        st.count[s] = 0;
        if (st.done[s]) continue;
        if (c > st.peak[s]) {
            st.peak[s] = c;
            st.peak_step[s] = t + 1;
        }
        if (c == 0) {
            st.length[s] = t + 1;
            st.done[s] = 1;
        } else {
            act = 1;
        }
    }
    act = __reduce_or_sync(FULL, act);
    if ((threadIdx.x & 31) == 0 && act) atomicAdd((unsigned long long *)(active + (t & 1)), 1ull);
}

// Simulations still running after the last step: truncated at `steps`.
__global__ void k_sir_close(int32_t B, int32_t steps, SirState st, uint8_t *__restrict__ truncated) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < B; s += gridDim.x * blockDim.x) {
        const bool tr = !st.done[s];
        if (tr) st.length[s] = steps;
        if (truncated) truncated[s] = tr;
    }
}

// Spreading power: an infected non-root node v is a descendant of its g-th
// ancestor at generation g; exact[g-1][anc] counts those, over simulations
// with final size >= min_size.  infected[v] counts those simulations in
// which v was infected.
__global__ void k_sir_tree(int32_t B, int32_t n, int32_t depth, int32_t min_size, SirState st,
                           unsigned long long *__restrict__ exact, unsigned long long *__restrict__ infected) {
    const int64_t total = (int64_t)B * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i / n), v = (int)(i - (int64_t)s * n);
        const int32_t *par = st.parent + (int64_t)s * n;
        if (par[v] < 0 || st.fsize[s] < min_size) continue;
        if (infected) atomicAdd(infected + v, 1ull);
        if (!exact) continue;
        int anc = v;
        for (int g = 0; g < depth; ++g) {
            const int p = par[anc];
            if (p == anc) break;
            atomicAdd(exact + (int64_t)g * n + p, 1ull);
            anc = p;
        }
    }
}

// spread[k-1][v] = sum over g <= k of exact[g-1][v], in place.
__global__ void k_sir_cumulate(int32_t n, int32_t depth, int64_t *__restrict__ spread) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (int g = 0; g < depth; ++g) {
            acc += spread[(int64_t)g * n + v];
            spread[(int64_t)g * n + v] = acc;
        }
    }
}

static inline unsigned grid_for(int64_t work, int per_block, int64_t cap) {
    int64_t g = (work + per_block - 1) / per_block;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_sir_init(const int32_t *index_cases, int32_t B, int32_t n, const uint8_t *immune, int32_t num_sets,
                    const int32_t *imm_set, const SirState &st, const Tune &t, cudaStream_t s) {
    k_sir_init<<<grid_for((int64_t)B * n, 256, (int64_t)t.num_sms * 32), 256, 0, s>>>(B, n, immune, num_sets,
                                                                                     imm_set, st);
    k_sir_seed<<<grid_for(B, 256, (int64_t)t.num_sms * 4), 256, 0, s>>>(index_cases, B, n, st);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_step(const int32_t *rp, const int32_t *ci, int32_t n, int32_t B, int32_t step, const SirStep &p,
                    const SirState &st, int64_t *active, const Tune &t, cudaStream_t s) {
    const int c = step & 1;
    uint64_t *cur = st.list[c], *nxt = st.list[c ^ 1];
    int64_t *ccur = st.list_count + c, *cnxt = st.list_count + (c ^ 1);
    k_sir_spread<<<t.num_sms * 8, 256, 0, s>>>(rp, ci, n, step, p, st, cur, ccur, nxt, cnxt);
    k_sir_spread_heavy<<<t.num_sms * 8, 256, 0, s>>>(rp, ci, n, step, p, st, nxt, cnxt);
    k_sir_commit<<<t.num_sms * 8, 256, 0, s>>>(n, st, nxt, cnxt);
    k_sir_stats<<<grid_for(B, 256, (int64_t)t.num_sms * 4), 256, 0, s>>>(B, step, st, ccur, active);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_close(int32_t B, int32_t steps, const SirState &st, uint8_t *truncated, const Tune &t,
                     cudaStream_t s) {
    k_sir_close<<<grid_for(B, 256, (int64_t)t.num_sms * 4), 256, 0, s>>>(B, steps, st, truncated);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_tree(int32_t B, int32_t n, int32_t depth, int32_t min_size, const SirState &st, int64_t *spread,
                    int64_t *infected, const Tune &t, cudaStream_t s) {
    k_sir_tree<<<grid_for((int64_t)B * n, 256, (int64_t)t.num_sms * 32), 256, 0, s>>>(
        B, n, depth, min_size, st, reinterpret_cast<unsigned long long *>(spread),
        reinterpret_cast<unsigned long long *>(infected));
    if (spread && depth > 0)
        k_sir_cumulate<<<grid_for(n, 256, (int64_t)t.num_sms * 32), 256, 0, s>>>(n, depth, spread);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
