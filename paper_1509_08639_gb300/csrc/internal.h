// internal.h -- device data layout shared by the kernels and the host runtime
// of the miner (not part of the public ABI; see include/mine.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mine.h"

namespace mine {

// Direction codes of the alignment (2 bits per cell, 16 cells per uint32).
enum : uint32_t { DIR_DIAG = 0, DIR_UP = 1, DIR_LEFT = 2 };

// Source-element flag bits (token IDs are < 2^30, so the two top bits are free).
constexpr uint32_t ELEM_FIRST = 1u << 31;   // first occurrence of this translation in U_i
constexpr uint32_t ELEM_END = 1u << 30;     // last translation of one source token
constexpr uint32_t ELEM_TOKEN = (1u << 30) - 1;

// device error word values (0 = fine)
constexpr int32_t ERR_DUP_KEY = 1;
constexpr int32_t ERR_BAD_OFFSETS = 2;
constexpr int32_t ERR_BAD_TOKEN = 3;

constexpr int kWarp = 32;
constexpr int kColHashLog2 = 11;            // per-warp target-token table, 2048 slots
constexpr int kColHashSlots = 1 << kColHashLog2;
constexpr int kColTokCap = kColHashSlots / 2;   // tokens per column block at most
constexpr int kPrepHashLog2 = 12;           // per-warp dedupe tables of the prep kernel
constexpr int kPrepHashSlots = 1 << kPrepHashLog2;
constexpr int kPrepElemCap = kPrepHashSlots / 2;
constexpr int kMaxSentTokens = MINE_MAX_SENT_TOKENS;

// Resident dictionary: open-addressed table of (key, off << 6 | cnt), linear
// probing, hash = key * 0x9E3779B1 >> (32 - log2).  Empty key = -1.
struct DevDict {
    int2 *slots;        // [1 << log2]
    int32_t *trans;     // translations
    int32_t log2;
    int32_t kmax;       // largest translation count of any key
    int64_t n_trans;
};

struct PairPlan {       // 48 bytes
    int32_t s0, S;      // source sentences [s0, s0+S) (global sentence index)
    int32_t t0, T;      // target sentences [t0, t0+T)
    int32_t set0, nset; // settings rows [set0, set0+nset)
    int32_t gap0, ngap; // distinct gaps [gap0, gap0+ngap) of this pair
    int64_t m_off;      // int32 offset of M (S rows, pitch Tp = round_up(T, 4))
    int64_t sel_base;   // mine_pair offset of the selection block (nset * min(S,T))
};

struct NwItem {         // one alignment: (pair, gap)
    int32_t pair;
    int32_t gap;        // global gap index
    int64_t code_off;   // uint32 offset of the direction codes (S rows x ceil(T/16) words)
    int64_t match_off;  // uint32 offset of the match list (min(S,T) entries)
    int64_t hrow_off;   // int32 offset of the row buffer (T+1 entries)
};

struct ScoreItem {      // 32 source rows of one pair
    int32_t pair;
    int32_t row0;
};

struct BatchDev {
    // inputs
    const int32_t *sent_off;     // [n_sent+1]
    const int32_t *tokens;       // [n_tok]
    int32_t n_pairs;
    // plan
    const PairPlan *pairs;
    const ScoreItem *score_items;
    int32_t n_score_items;
    const NwItem *nw_items;
    int32_t n_nw_items;
    const int32_t *set_gap;      // [R] global gap index of each setting row
    const int32_t *set_thr;      // [R]
    const int32_t *gap_val;      // [G]
    // scratch
    uint32_t *elems;             // [n_tok * kmax]
    int4 *sinfo;                 // [n_sent] (n_i, n_elem, |U_i|, 0) for source sentences
    int32_t *M;                  // scores
    uint32_t *codes;             // directions
    uint32_t *matches;           // traceback matches (i << 16 | j), decreasing i
    int32_t *hrow;               // alignment row buffers
    int32_t *counters;           // [4] work-queue heads
    int32_t *err;                // error word (0 = fine)
    // outputs
    int32_t *nw_score;           // [R]
    int32_t *n_sel;              // [R]
    int32_t *sel;                // mine_pair triples
};

// launchers (kernels.cu); each returns the number of kernels launched
int launch_dict_build(const int32_t *keys, const int32_t *trans_off, int32_t n_keys, DevDict d,
                      int32_t *err, cudaStream_t st);
int launch_validate(const int32_t *sent_off, int64_t n_sent, int64_t n_tok, int32_t *err,
                    cudaStream_t st);
int launch_prep(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st);
int launch_score(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st);

// kernel identities for per-kernel timing
enum KernelId { KID_DICT = 0, KID_VALIDATE = 1, KID_PREP = 2, KID_SCORE = 3, KID_ALIGN = 4,
                KID_COUNT = 5 };
int launch_align(const BatchDev &b, int num_sms, cudaStream_t st);
int launch_compact(const int32_t *src, const int64_t *src_off, const int64_t *dst_off,
                   const int32_t *counts, int32_t n_rows, int32_t *dst, cudaStream_t st);

}  // namespace mine
