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
// Layout, node-major: a batch of B <= SIR_BATCH simulations runs together,
// and each node keeps WB = ceil(B / 32) words of one bit per simulation:
// susceptible, infected at the start of the step (inf[cur]), infected at the
// start of the next (inf[nxt]), and infected during this step (newinf).  A
// node infected in any simulation is in the step's frontier once; its
// neighbour list is read once for all simulations, and for a neighbour x
// the words inf[cur][u] & susc[x] say which simulations try the edge, the
// words read by consecutive lanes.  cand (node-major, x * B + s) holds the
// smallest successful infector of the step, parent (simulation-major, the
// output layout) the infection tree.  Kernels of a step:
//   k_sir_spread        a warp per frontier node: recovery draws (slot 0),
//                       then (slot, word) lanes over the neighbours; nodes
//                       of degree > SIR_HEAVY are listed for
//   k_sir_spread_heavy  a CTA per listed node over its neighbours
//   k_sir_commit        per node with a success: new infections, parents
//   k_sir_clear         zeroes the frontier's inf[cur] words for reuse
//   k_sir_stats         per simulation: peak, its step, length
// Lists are deduplicated by per-node step stamps, per-simulation counts are
// summed in shared memory per block, and the host reads whether any
// simulation is still running every SIR_CHECK steps.
#include "ef_internal.cuh"

namespace ef {

constexpr int32_t NO_CAND = 0x7fffffff;
constexpr uint32_t RECOVER_WORD = 0xffffffffu;
constexpr int SIR_HEAVY = 256;   // frontier nodes of higher degree take a CTA each

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

// Lane geometry of a warp over (slot, word) pairs: wbp = WB rounded up to a
// power of two, 32 / wbp slots (nodes or neighbours) per warp.
struct SirLanes {
    int wbp, slots, slot, w;
    bool wv;
    __device__ __forceinline__ explicit SirLanes(int WB) {
        wbp = 1;
        while (wbp < WB) wbp <<= 1;
        slots = 32 / wbp;
        const int lane = threadIdx.x & 31;
        slot = lane / wbp;
        w = lane % wbp;
        wv = w < WB;
    }
};

// Append v to list (count *cnt) unless it was appended with this stamp.
__device__ __forceinline__ void sir_append(int32_t *list, int32_t *cnt, int32_t *mark, int v, int stamp) {
    if (atomicExch(mark + v, stamp) != stamp) list[atomicAdd(cnt, 1)] = v;
}

__global__ void k_sir_fill(int32_t *__restrict__ a, int64_t len, int32_t value) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = value;
}

// Susceptibility words: every simulation but those whose immune set holds v.
__global__ void k_sir_init_susc(int32_t n, const uint8_t *__restrict__ immune, int32_t num_sets,
                                const int32_t *__restrict__ imm_set, SirState st) {
    const int64_t words = (int64_t)n * st.WB;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / st.WB), w = (int)(i - (int64_t)v * st.WB);
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int s = w * 32 + b;
            if (s >= st.B) break;
            int set = imm_set ? imm_set[s] : -1;
            if (set >= num_sets) {
                atomicOr(st.err, ERRB_SIR_ARG);
                set = -1;
            }
            if (set < 0 || !immune[(int64_t)set * n + v]) word |= 1u << b;
        }
        st.susc[i] = word;
    }
}

// The index cases and the first frontier (an immune index case is an error).
__global__ void k_sir_seed(const int32_t *__restrict__ index_cases, int32_t n, SirState st) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < st.B; s += gridDim.x * blockDim.x) {
        const int u = index_cases[s];
        st.peak[s] = 1;
        st.peak_step[s] = 0;
        st.length[s] = 0;
        st.count[s] = 1;
        st.fsize[s] = 1;
        st.done[s] = 0;
        const uint32_t bit = 1u << (s & 31);
        if (u < 0 || u >= n || !(st.susc[(int64_t)u * st.WB + (s >> 5)] & bit)) {
            atomicOr(st.err, ERRB_SIR_ARG);
            st.done[s] = 1;
            st.count[s] = 0;
            st.fsize[s] = 0;
            continue;
        }
        atomicAnd(st.susc + (int64_t)u * st.WB + (s >> 5), ~bit);   // index cases may share a node
        atomicOr(st.inf[0] + (int64_t)u * st.WB + (s >> 5), bit);
        st.parent[(int64_t)s * n + u] = u;
        sir_append(st.front[0], st.counts + 0, st.fmark, u, -1);
    }
}

// Tries of u's infected simulations (its inf[cur] words iw) over the
// neighbours k_first, k_first + stride, ... (the warp's slots taking
// consecutive neighbours).
// The loads of SIR_UNROLL neighbours are issued before any of their tries.
constexpr int SIR_UNROLL = 4;
__device__ __forceinline__ void sir_tries(const int32_t *__restrict__ ci, int a, int D, int u, int t, uint32_t iw,
                                          const SirLanes &L, int k_first, int stride, const SirStep &p,
                                          const SirState &st) {
    for (int k0 = k_first; k0 < D; k0 += SIR_UNROLL * stride) {
        int x[SIR_UNROLL];
        uint32_t act[SIR_UNROLL];
#pragma unroll
        for (int q = 0; q < SIR_UNROLL; ++q) {
            const int k = k0 + q * stride + L.slot;
            x[q] = k < D ? ci[a + k] : -1;
        }
#pragma unroll
        for (int q = 0; q < SIR_UNROLL; ++q)
            act[q] = x[q] >= 0 && L.wv ? iw & st.susc[(int64_t)x[q] * st.WB + L.w] : 0u;
#pragma unroll
        for (int q = 0; q < SIR_UNROLL; ++q) {
            uint32_t m = act[q];
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int s = L.w * 32 + b;
                const uint32_t r =
                    philox_w0((uint32_t)(p.sim_base + s), (uint32_t)t, (uint32_t)u, (uint32_t)x[q], p.seed);
                if ((uint64_t)r < p.beta_thr && atomicMin(st.cand + (int64_t)x[q] * st.B + s, u) == NO_CAND) {
                    atomicOr(st.newinf + (int64_t)x[q] * st.WB + L.w, 1u << b);
                    sir_append(st.touched, st.counts + 2, st.tmark, x[q], t + 1);
                }
            }
        }
    }
}

// One step over the frontier front[cur]: recoveries, survivors into
// inf[nxt] and front[nxt], tries of the nodes of degree <= SIR_HEAVY.
__global__ void __launch_bounds__(256) k_sir_spread(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                    int32_t t, SirStep p, SirState st) {
    __shared__ int s_rec[SIR_BATCH];
    for (int i = threadIdx.x; i < st.B; i += blockDim.x) s_rec[i] = 0;
    __syncthreads();
    const int c = t & 1, nx = c ^ 1, lane = threadIdx.x & 31;
    const SirLanes L(st.WB);
    const int total = st.counts[c];
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < total; i += nwarps) {
        const int u = st.front[c][i];
        const int a = rp[u], D = rp[u + 1] - a;
        const uint32_t iw = L.wv ? st.inf[c][(int64_t)u * st.WB + L.w] : 0u;
        uint32_t sv = iw;
        if (L.slot == 0 && L.wv) {
            uint32_t m = iw;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int s = L.w * 32 + b;
                const uint32_t r =
                    philox_w0((uint32_t)(p.sim_base + s), (uint32_t)t, (uint32_t)u, RECOVER_WORD, p.seed);
                if ((uint64_t)r < p.gamma_thr) {
                    sv &= ~(1u << b);
                    atomicAdd(s_rec + s, 1);
                }
            }
            st.inf[nx][(int64_t)u * st.WB + L.w] = sv;
        }
        const bool survives = __any_sync(FULL, L.slot == 0 && sv != 0u);
        if (survives && lane == 0) sir_append(st.front[nx], st.counts + nx, st.fmark, u, t + 1);
        if (D > SIR_HEAVY) {
            if (lane == 0) st.heavy[atomicAdd(st.counts + 3, 1)] = u;
            continue;
        }
        sir_tries(ci, a, D, u, t, iw, L, 0, L.slots, p, st);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < st.B; s += blockDim.x)
        if (s_rec[s]) atomicSub(st.count + s, s_rec[s]);
}

__global__ void __launch_bounds__(256) k_sir_spread_heavy(const int32_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci, int32_t t, SirStep p,
                                                          SirState st) {
    const int c = t & 1, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const SirLanes L(st.WB);
    const int total = st.counts[3];
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const int u = st.heavy[i];
        const int a = rp[u], D = rp[u + 1] - a;
        const uint32_t iw = L.wv ? st.inf[c][(int64_t)u * st.WB + L.w] : 0u;
        sir_tries(ci, a, D, u, t, iw, L, wid * L.slots, nw * L.slots, p, st);
    }
}

// New infections of the step: per node with a success, its newinf words.
__global__ void __launch_bounds__(256) k_sir_commit(int32_t n, int32_t t, SirState st) {
    __shared__ int s_new[SIR_BATCH];
    for (int i = threadIdx.x; i < st.B; i += blockDim.x) s_new[i] = 0;
    __syncthreads();
    const int nx = (t & 1) ^ 1;
    const SirLanes L(st.WB);
    const int total = st.counts[2];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned mine = (L.wbp == 32 ? FULL : (1u << L.wbp) - 1u) << (L.slot * L.wbp);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * L.slots; base < total;
         base += nwarps * L.slots) {
        const int64_t i = base + L.slot;
        const int x = i < total ? st.touched[i] : -1;
        uint32_t nb = 0;
        if (x >= 0 && L.wv) {
            const int64_t j = (int64_t)x * st.WB + L.w;
            nb = st.newinf[j];
            if (nb) {
                st.newinf[j] = 0;
                st.susc[j] &= ~nb;
                st.inf[nx][j] |= nb;
                uint32_t m = nb;
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const int s = L.w * 32 + b;
                    int32_t *cs = st.cand + (int64_t)x * st.B + s;
                    st.parent[(int64_t)s * n + x] = *cs;
                    *cs = NO_CAND;
                    atomicAdd(s_new + s, 1);
                }
            }
        }
        // the node joins the next frontier once (it may already be there as a survivor)
        const unsigned any = __ballot_sync(FULL, nb != 0u);
        if (L.w == 0 && (any & mine)) sir_append(st.front[nx], st.counts + nx, st.fmark, x, t + 1);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < st.B; s += blockDim.x)
        if (s_new[s]) {
            atomicAdd(st.count + s, s_new[s]);
            atomicAdd(st.fsize + s, s_new[s]);
        }
}

// The frontier's words of inf[cur], zeroed: the buffer is the next step's inf[nxt].
__global__ void k_sir_clear(int32_t t, SirState st) {
    const int c = t & 1;
    const int64_t total = (int64_t)st.counts[c] * st.WB;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = st.front[c][i / st.WB];
        st.inf[c][(int64_t)v * st.WB + (i % st.WB)] = 0u;
    }
}

// After step t: count[s] = infected at the start of step t + 1.  active[t & 1]
// counts warps with a simulation still running; the emptied lists and
// active[(t + 1) & 1] are cleared for the next step.
__global__ void k_sir_stats(int32_t t, SirState st, int64_t *__restrict__ active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st.counts[t & 1] = 0;
        st.counts[2] = 0;
        st.counts[3] = 0;
        active[(t + 1) & 1] = 0;
    }
    int act = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < st.B; s += gridDim.x * blockDim.x) {
        if (st.done[s]) continue;
        const int cnt = st.count[s];
        if (cnt > st.peak[s]) {
            st.peak[s] = cnt;
            st.peak_step[s] = t + 1;
        }
        if (cnt == 0) {
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
__global__ void k_sir_close(int32_t steps, SirState st, uint8_t *__restrict__ truncated) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < st.B; s += gridDim.x * blockDim.x) {
        const bool tr = !st.done[s];
        if (tr) st.length[s] = steps;
        if (truncated) truncated[s] = tr;
    }
}

// Spreading power: an infected non-root node v is a descendant of its g-th
// ancestor at generation g; exact[g-1][anc] counts those, over simulations
// with final size >= min_size.  infected[v] counts those simulations in
// which v was infected.
__global__ void k_sir_tree(int32_t n, int32_t depth, int32_t min_size, SirState st,
                           unsigned long long *__restrict__ exact, unsigned long long *__restrict__ infected) {
    const int64_t total = (int64_t)st.B * n;
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

int launch_sir_init(const int32_t *index_cases, int32_t n, const uint8_t *immune, int32_t num_sets,
                    const int32_t *imm_set, const SirState &st, const Tune &t, cudaStream_t s) {
    const int64_t cap = (int64_t)t.num_sms * 32, nb = (int64_t)n * st.B;
    k_sir_fill<<<grid_for(nb, 256, cap), 256, 0, s>>>(st.cand, nb, NO_CAND);
    k_sir_fill<<<grid_for(nb, 256, cap), 256, 0, s>>>(st.parent, nb, -1);
    k_sir_init_susc<<<grid_for((int64_t)n * st.WB, 256, cap), 256, 0, s>>>(n, immune, num_sets, imm_set, st);
    k_sir_seed<<<grid_for(st.B, 256, cap), 256, 0, s>>>(index_cases, n, st);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_step(const int32_t *rp, const int32_t *ci, int32_t n, int32_t step, const SirStep &p,
                    const SirState &st, int64_t *active, const Tune &t, cudaStream_t s) {
    const unsigned g = (unsigned)t.num_sms * 8;
    k_sir_spread<<<g, 256, 0, s>>>(rp, ci, step, p, st);
    k_sir_spread_heavy<<<g, 256, 0, s>>>(rp, ci, step, p, st);
    k_sir_commit<<<g, 256, 0, s>>>(n, step, st);
    k_sir_clear<<<g, 256, 0, s>>>(step, st);
    k_sir_stats<<<grid_for(st.B, 256, (int64_t)t.num_sms * 4), 256, 0, s>>>(step, st, active);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_close(int32_t steps, const SirState &st, uint8_t *truncated, const Tune &t, cudaStream_t s) {
    k_sir_close<<<grid_for(st.B, 256, (int64_t)t.num_sms * 4), 256, 0, s>>>(steps, st, truncated);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_tree(int32_t n, int32_t depth, int32_t min_size, const SirState &st, int64_t *exact,
                    int64_t *infected, const Tune &t, cudaStream_t s) {
    k_sir_tree<<<grid_for((int64_t)st.B * n, 256, (int64_t)t.num_sms * 32), 256, 0, s>>>(
        n, depth, min_size, st, reinterpret_cast<unsigned long long *>(exact),
        reinterpret_cast<unsigned long long *>(infected));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sir_cumulate(int32_t n, int32_t depth, int64_t *spread, const Tune &t, cudaStream_t s) {
    k_sir_cumulate<<<grid_for(n, 256, (int64_t)t.num_sms * 32), 256, 0, s>>>(n, depth, spread);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
