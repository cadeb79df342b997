// DL0 byte-stream ingest (Sec. 5: telescope data as a telemetry-formatted byte
// stream; the packet layout is documented in include/rta.h). The decoder builds
// a directory of the stream -- segments, images, events -- and copies nothing:
// the image kernel reads each chunk of pixels from the segment that holds it.
//
// Framing: packets follow one another and only a walk from byte 0 knows where
// they start. The stream is cut into 1 MiB pieces. Each piece looks for its
// first valid packet (16-byte aligned positions, a header whose fields hold and
// whose successor's header holds too; 256 positions per round) and walks from
// there to the end of the piece. The walks must join up: piece b's first packet
// is where piece b-1's walk ended. Where they do not (a fault, or a payload that
// happens to look like a header) a single thread walks on from the last joined
// position, and the piece counts are redone from that walk.
//
// Checks: every packet gets the oracle's checks in the oracle's order (framing,
// fixed header fields, camera, segment order, CRC, capacity); the fault reported
// is the one of the earliest packet. The CRC (optional) is computed per packet
// by a warp: each lane four pieces, four bytes per step with four lookup
// tables, and the pieces combined in GF(2)[x] modulo the generator.
#include <algorithm>

#include "rta_launch.cuh"

namespace rta {

namespace {

constexpr int64_t ING_CHUNK = int64_t(1) << 20;
constexpr int ING_SCAN_THREADS = 256;

struct PktFields {
    int apid, seq_flags, length, first, n, P, S;
    uint32_t sec, fine;
    uint64_t event;
};

__device__ __forceinline__ uint32_t byte_of(const uint4& a, const uint4& b, int i) {
    const uint4& v = i < 16 ? a : b;
    const int j = i & 15;
    const uint32_t w = j < 4 ? v.x : j < 8 ? v.y : j < 12 ? v.z : v.w;
    return (w >> (8 * (j & 3))) & 0xFFu;
}

__device__ __forceinline__ uint32_t be16(const uint4& a, const uint4& b, int i) {
    return (byte_of(a, b, i) << 8) | byte_of(a, b, i + 1);
}

__device__ __forceinline__ uint32_t be32(const uint4& a, const uint4& b, int i) {
    return (be16(a, b, i) << 16) | be16(a, b, i + 2);
}

// The oracle's framing, header and camera checks of the packet at pos (16-byte
// aligned), in its order; fills f when the header could be read.
__device__ int pkt_check(const uint8_t* s, int64_t pos, int64_t n_bytes, const DevArray& arr, PktFields& f) {
    if (n_bytes - pos < 48) return RTA_STREAM_FRAMING;
    const uint4* h = reinterpret_cast<const uint4*>(s + pos);
    const uint4 a = __ldg(h), b = __ldg(h + 1);
    const uint32_t w0 = be16(a, b, 0), w1 = be16(a, b, 2);
    f.apid = int(w0 & 0x7FFu);
    f.seq_flags = int(w1 >> 14);
    f.length = int(be16(a, b, 4)) + 7;
    f.sec = be32(a, b, 10);
    f.fine = be16(a, b, 14);
    f.event = (uint64_t(be32(a, b, 16)) << 32) | be32(a, b, 20);
    f.first = int(be16(a, b, 24));
    f.n = int(be16(a, b, 26));
    f.P = int(be16(a, b, 28));
    f.S = int(be16(a, b, 30));
    if ((w0 >> 13) != 0 || ((w0 >> 12) & 1u) != 0 || ((w0 >> 11) & 1u) != 1 || byte_of(a, b, 6) != 0x10 ||
        byte_of(a, b, 7) != RTA_PKT_SERVICE || byte_of(a, b, 8) != RTA_PKT_SUBSERVICE)
        return RTA_STREAM_HEADER;
    const int L = f.length;
    if ((L & 15) || L < 48 || L > RTA_PKT_MAX_BYTES || pos + L > n_bytes) return RTA_STREAM_FRAMING;
    if (48 + 2 * f.n * f.S != L || f.n == 0 || ((f.n * f.S) & 7) || f.first + f.n > f.P) return RTA_STREAM_HEADER;
    const bool starts = f.first == 0, ends = f.first + f.n == f.P;
    const int want = starts && ends ? 3 : starts ? 1 : ends ? 2 : 0;
    if (f.seq_flags != want) return RTA_STREAM_HEADER;
    if (f.apid >= arr.n_tel) return RTA_STREAM_CAMERA;
    const DevCam& C = arr.cams[arr.tel_cam[f.apid]];
    if (C.P != f.P || C.S != f.S) return RTA_STREAM_CAMERA;
    return RTA_STREAM_OK;
}

// A position where a packet can start: its checks hold and so do its successor's.
__device__ __forceinline__ bool plausible_start(const uint8_t* s, int64_t pos, int64_t n_bytes, const DevArray& arr) {
    PktFields f, g;
    if (pkt_check(s, pos, n_bytes, arr, f) != RTA_STREAM_OK) return false;
    const int64_t nx = pos + f.length;
    return nx == n_bytes || pkt_check(s, nx, n_bytes, arr, g) == RTA_STREAM_OK;
}

}  // namespace

__global__ void k_ingest_init(const IngestArgs a) { a.hdr->first_bad_pk = LLONG_MAX; }

// ---------------------------------------------------------------- framing
// One block per piece: its first plausible packet start, then the walk.
__global__ void __launch_bounds__(ING_SCAN_THREADS) k_frame_scan(const IngestArgs a) {
    __shared__ long long found;
    const int64_t b = blockIdx.x;
    const int64_t c0 = b * ING_CHUNK, c1 = c0 + ING_CHUNK < a.n_bytes ? c0 + ING_CHUNK : a.n_bytes;
    if (threadIdx.x == 0) found = b == 0 ? 0 : LLONG_MAX;
    __syncthreads();
    if (b > 0) {
        for (int64_t r0 = c0; r0 < c1; r0 += 16 * ING_SCAN_THREADS) {
            const int64_t pos = r0 + 16 * int64_t(threadIdx.x);
            if (pos < c1 && plausible_start(a.stream, pos, a.n_bytes, a.arr)) atomicMin(&found, (long long)pos);
            __syncthreads();
            if (found != LLONG_MAX) break;
        }
    }
    if (threadIdx.x != 0) return;
    IngChunk ch = {};
    ch.err = 0;
    ch.err_pos = -1;
    if (found == LLONG_MAX) {
        ch.first = -1;
        ch.end = -1;
        a.chunks[b] = ch;
        return;
    }
    ch.first = found;
    int64_t pos = found;
    int count = 0;
    while (pos < c1) {
        PktFields f;
        const int code = pkt_check(a.stream, pos, a.n_bytes, a.arr, f);
        if (code != RTA_STREAM_OK) {
            ch.err = code;
            ch.err_pos = pos;
            break;
        }
        ++count;
        pos += f.length;
    }
    ch.count = count;
    ch.end = pos;
    a.chunks[b] = ch;
}

// Joins the walks (one block). The walks are on the true chain up to the first
// piece whose first packet is not where the previous walk ended; from there one
// thread walks on and rewrites the pieces' starts and counts, stopping at the
// first framing/header/camera fault. Then an exclusive scan of the counts.
__global__ void __launch_bounds__(1024) k_frame_join(const IngestArgs a) {
    __shared__ long long first_bad;
    const int64_t nc = a.n_chunks;
    if (threadIdx.x == 0) first_bad = LLONG_MAX;
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nc; b += blockDim.x) {
        const IngChunk& ch = a.chunks[b];
        bool bad = ch.first < 0 || ch.err != 0;
        if (b > 0) bad = bad || ch.first != a.chunks[b - 1].end;
        if (bad) atomicMin(&first_bad, (long long)b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t fb = first_bad;
        a.hdr->walk_err = 0;
        a.hdr->walk_err_pos = -1;
        if (fb != LLONG_MAX) {
            // the true chain is known up to the start of piece fb
            int64_t pos = fb == 0 ? 0 : a.chunks[fb - 1].end;
            for (int64_t b = fb; b < nc; ++b) {
                IngChunk ch = {};
                const int64_t c1 = (b + 1) * ING_CHUNK < a.n_bytes ? (b + 1) * ING_CHUNK : a.n_bytes;
                ch.first = pos;
                int count = 0;
                while (pos < c1) {
                    PktFields f;
                    const int code = pkt_check(a.stream, pos, a.n_bytes, a.arr, f);
                    if (code != RTA_STREAM_OK) {
                        a.hdr->walk_err = code;
                        a.hdr->walk_err_pos = pos;
                        break;
                    }
                    ++count;
                    pos += f.length;
                }
                ch.count = count;
                ch.end = pos;
                a.chunks[b] = ch;
                if (a.hdr->walk_err) {
                    for (int64_t r = b + 1; r < nc; ++r) a.chunks[r].count = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    // exclusive scan of the pieces' packet counts, 1024 pieces at a time
    __shared__ long long wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t0 = 0; t0 < nc; t0 += blockDim.x) {
        const int64_t b = t0 + threadIdx.x;
        const long long v = b < nc ? a.chunks[b].count : 0;
        long long incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            long long w = lane < int(blockDim.x >> 5) ? wsum[lane] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            wsum[lane] = w;              // inclusive over warps
        }
        __syncthreads();
        const long long before = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - v;
        if (b < nc) a.chunks[b].base = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.hdr->n_pk = carry;
}

// One block per piece: the packets' offsets (the first seg_cap + 1 of them).
__global__ void __launch_bounds__(32) k_frame_list(const IngestArgs a) {
    if (threadIdx.x != 0) return;
    const IngChunk ch = a.chunks[blockIdx.x];
    int64_t pos = ch.first;
    for (int j = 0; j < ch.count; ++j) {
        const int64_t k = ch.base + j;
        if (k > a.seg_cap) break;
        a.pk_off[k] = pos;
        PktFields f;
        pkt_check(a.stream, pos, a.n_bytes, a.arr, f);
        pos += f.length;
    }
}

// ---------------------------------------------------------------- per-packet checks
// Segment order, and the scan values: image start (high word), event start (low).
__global__ void __launch_bounds__(256) k_pkt_check(const IngestArgs a) {
    const int64_t n = a.hdr->n_pk < a.seg_cap + 1 ? a.hdr->n_pk : a.seg_cap + 1;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        PktFields f;
        pkt_check(a.stream, a.pk_off[k], a.n_bytes, a.arr, f);     // passed in the walk
        int err = 0;
        bool new_event = f.first == 0;
        if (k > 0) {
            PktFields g;
            pkt_check(a.stream, a.pk_off[k - 1], a.n_bytes, a.arr, g);
            if (g.first + g.n < g.P) {
                if (f.apid != g.apid || f.event != g.event || f.first != g.first + g.n) err = RTA_STREAM_SEGMENT;
            } else if (f.first != 0) {
                err = RTA_STREAM_SEGMENT;
            }
            new_event = new_event && f.event != g.event;
        } else if (f.first != 0) {
            err = RTA_STREAM_SEGMENT;
        }
        // the stream may not end inside an image (only when the walk reached the end)
        if (!err && k == a.hdr->n_pk - 1 && !a.hdr->walk_err && f.first + f.n < f.P) err = RTA_STREAM_SEGMENT;
        a.pk_err[k] = err;
        a.pk_scan[k] = (uint64_t(f.first == 0) << 32) | uint64_t(new_event);
    }
}

// ---------------------------------------------------------------- CRC
namespace {

// Product of two polynomials of degree < 16 modulo x^16 + x^12 + x^5 + 1.
__device__ __forceinline__ uint32_t gf_mulmod(uint32_t x, uint32_t y) {
    uint32_t p = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if ((y >> i) & 1u) p ^= x << i;
#pragma unroll
    for (int i = 30; i >= 16; --i)
        if ((p >> i) & 1u) p ^= 0x11021u << (i - 16);
    return p & 0xFFFFu;
}

__device__ __forceinline__ uint32_t gf_pow(uint32_t b, int e) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = gf_mulmod(r, b);
        b = gf_mulmod(b, b);
        e >>= 1;
    }
    return r;
}

constexpr int CRC_X16 = RTA_PKT_MAX_BYTES / 16 + 1;
constexpr int CRC_THREADS = 1024;                 // one CTA per SM (the lane tables fill most of its shared memory)
constexpr int CRC_STRIDE_WORDS = 32;             // a lane's 16-byte words are this far apart
constexpr size_t CRC_LANE_TABLE_BYTES = size_t(6) * 256 * 32 * 4;
constexpr size_t CRC_SMEM_BYTES =
    CRC_LANE_TABLE_BYTES + 2 * (size_t(6) * 256 + CRC_X16 + 64 + CRC_X16 / 64 + 1);
static_assert(CRC_SMEM_BYTES <= 227 * 1024, "shared memory per CTA");

}  // namespace

// One warp per packet. For a correct packet, running the CRC register over all
// L bytes -- the CRC field included, most significant byte first -- ends at 0
// (the register after the message equals the field, and two bytes equal to the
// register clear it). The register is linear in the message, so the packet's
// 16-byte words can be taken in any grouping: lane l takes words l, l + 32, ...
// (the warp reads 512 contiguous bytes a step), forms each word's CRC from a zero
// register (four bytes a step through four lookup tables) and folds it into its
// own register, which is carried over the 512-byte stride between its words by
// two more tables (multiplication by x^4096 modulo the generator). At the end
// each lane's register is carried to the packet's end by x^(8 k), k the bytes
// after its last word, from a table over multiples of 16 bytes; the preset
// register 0xFFFF is carried likewise; the XOR of all of it must be 0. Every
// lane has its own copy of the tables in shared memory, so a warp's lookups hit
// 32 different banks.
__global__ void __launch_bounds__(CRC_THREADS, 1) k_pkt_crc(const IngestArgs a) {
    extern __shared__ __align__(16) unsigned char crc_smem[];
    uint16_t* T = reinterpret_cast<uint16_t*>(crc_smem + CRC_LANE_TABLE_BYTES); // [6][256]
    uint16_t* X16 = T + 6 * 256;                                                // x^(128 k) mod G
    uint16_t* A = X16 + CRC_X16;
    uint16_t* B = A + 64;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint32_t r = uint32_t(i) << 8;
        for (int k = 0; k < 8; ++k) r = (r & 0x8000u) ? ((r << 1) ^ 0x1021u) : (r << 1);
        T[i] = uint16_t(r);
    }
    const uint32_t x128 = gf_pow(2u, 128);          // x^128 = 16 zero bytes
    if (threadIdx.x < 64) A[threadIdx.x] = uint16_t(gf_pow(x128, threadIdx.x));
    if (threadIdx.x < CRC_X16 / 64 + 1) B[threadIdx.x] = uint16_t(gf_pow(gf_pow(x128, 64), threadIdx.x));
    __syncthreads();
    const uint32_t K = gf_pow(2u, 8 * 16 * CRC_STRIDE_WORDS);     // one lane's stride: 32 words
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        // T[k][x]: byte x followed by k zero bytes, register starting at zero
        uint32_t r = T[i];
        for (int k = 1; k < 4; ++k) {
            r = ((r << 8) & 0xFFFFu) ^ T[(r >> 8) & 0xFFu];
            T[k * 256 + i] = uint16_t(r);
        }
        // register (x : 0) and (0 : x) carried over one lane stride of zero bytes
        T[4 * 256 + i] = uint16_t(gf_mulmod(uint32_t(i) << 8, K));
        T[5 * 256 + i] = uint16_t(gf_mulmod(uint32_t(i), K));
    }
    for (int k = threadIdx.x; k < CRC_X16; k += blockDim.x) X16[k] = uint16_t(gf_mulmod(A[k & 63], B[k >> 6]));
    __syncthreads();
    // one copy of the six tables per lane: entry (k, x) of lane l at byte
    // 65536 (k >> 1) + 256 x + 128 (k & 1) + 4 l, so that every lookup of a warp hits
    // 32 different banks and a lookup's offset is one byte permute of the index
    // byte and 4 l (the table's constant part goes into the load's immediate)
    for (int w = threadIdx.x; w < 6 * 256 * 32; w += blockDim.x) {
        const int k = w >> 13, x = (w >> 5) & 255, l = w & 31;
        *reinterpret_cast<uint32_t*>(crc_smem + 65536 * (k >> 1) + 256 * x + 128 * (k & 1) + 4 * l) = T[k * 256 + x];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t l4 = uint32_t(lane) * 4u;
    // entry of table k at the index in byte j of v (byte permute: l4 in byte 0, the
    // index byte in byte 1, zeros above)
    auto look = [&](int k, uint32_t v, int j) {
        const uint32_t off = __byte_perm(v, l4, 0x7604u | (uint32_t(j) << 4));
        return *reinterpret_cast<const uint32_t*>(crc_smem + off + 65536 * (k >> 1) + 128 * (k & 1));
    };
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t n = a.hdr->n_pk < a.seg_cap + 1 ? a.hdr->n_pk : a.seg_cap + 1;
    for (int64_t k = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n; k += warps) {
        const int64_t pos = a.pk_off[k];
        const uint4* p = reinterpret_cast<const uint4*>(a.stream + pos);
        PktFields f;
        pkt_check(a.stream, pos, a.n_bytes, a.arr, f);
        const int L = f.length;                           // multiple of 16
        const int words = L >> 4;
        // lane l takes words l, l + 32, ...: one coalesced 512-byte load per warp and
        // step, issued one step ahead. Its register r covers its words with zeros
        // between them: r <- r x^(8 * 512) + CRC_0(word), the word's own CRC from a
        // zero register.
        uint32_t r = 0;
        int w = lane;
        uint4 qn = w < words ? __ldg(p + w) : make_uint4(0, 0, 0, 0);
        int last = -1;
        for (; w < words; w += CRC_STRIDE_WORDS) {
            const uint4 q = qn;
            if (w + CRC_STRIDE_WORDS < words) qn = __ldg(p + w + CRC_STRIDE_WORDS);
            const uint32_t ws[4] = {q.x, q.y, q.z, q.w};
            uint32_t c = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t x = ws[j];
                const uint32_t u = c ^ __byte_perm(x, 0u, 0x4401u);     // register ^ (b0 : b1)
                c = look(3, u, 1) ^ look(2, u, 0) ^ look(1, x, 2) ^ look(0, x, 3);
            }
            r = look(4, r, 1) ^ look(5, r, 0) ^ c;
            last = w;
        }
        // carried to the packet's end; the preset register 0xFFFF likewise
        uint32_t v = last >= 0 ? gf_mulmod(r, X16[words - 1 - last]) : 0u;
        if (lane == 0) v ^= gf_mulmod(0xFFFFu, X16[words]);
        for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0 && a.pk_err[k] == 0) a.pk_err[k] = RTA_STREAM_CRC;
    }
}

// ---------------------------------------------------------------- scan of the packets' start flags
// Inclusive scan of 64-bit values (image starts in the high word, event starts
// in the low word) in blocks of 1024, then the blocks' offsets.
__global__ void __launch_bounds__(1024) k_pkt_scan_local(const IngestArgs a) {
    __shared__ unsigned long long wsum[32];
    const int64_t n = a.hdr->n_pk < a.seg_cap + 1 ? a.hdr->n_pk : a.seg_cap + 1;
    const int64_t k = int64_t(blockIdx.x) * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long v = k < n ? a.pk_scan[k] : 0ull;
    unsigned long long incl = v;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = wsum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    incl += warp > 0 ? wsum[warp - 1] : 0ull;
    if (k < n) a.pk_scan[k] = incl;
    if (threadIdx.x == 1023) a.blk_sum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) k_pkt_scan_blocks(const IngestArgs a, int64_t n_blk) {
    // one block: exclusive offsets of the blocks, 1024 at a time
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < n_blk; t0 += 1024) {
        const int64_t b = t0 + threadIdx.x;
        const unsigned long long v = b < n_blk ? a.blk_sum[b] : 0ull;
        unsigned long long incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = wsum[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp > 0 ? wsum[warp - 1] : 0ull) + incl - v;
        if (b < n_blk) a.blk_sum[b] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
}

// Adds the block offsets; then capacities, and the earliest faulty packet.
__global__ void __launch_bounds__(1024) k_pkt_final(const IngestArgs a) {
    const int64_t n = a.hdr->n_pk < a.seg_cap + 1 ? a.hdr->n_pk : a.seg_cap + 1;
    const int64_t k = int64_t(blockIdx.x) * 1024 + threadIdx.x;
    if (k >= n) return;
    const unsigned long long incl = a.pk_scan[k] + a.blk_sum[blockIdx.x];
    a.pk_scan[k] = incl;
    const int64_t img = int64_t(incl >> 32) - 1, evt = int64_t(incl & 0xFFFFFFFFull) - 1;
    int err = a.pk_err[k];
    if (!err && (k >= a.seg_cap || img >= a.img_cap || evt >= a.evt_cap)) err = RTA_STREAM_CAPACITY;
    a.pk_err[k] = err;
    if (err) atomicMin(reinterpret_cast<unsigned long long*>(&a.hdr->first_bad_pk), (unsigned long long)k);
}

// The verdict (one thread): the earliest faulty packet, else the walk's fault.
__global__ void k_ingest_verdict(const IngestArgs a) {
    IngHdr& h = *a.hdr;
    const int64_t n = h.n_pk < a.seg_cap + 1 ? h.n_pk : a.seg_cap + 1;
    int64_t* c = a.counts;
    int err = 0;
    int64_t pos = -1;
    if (h.first_bad_pk < n) {
        err = a.pk_err[h.first_bad_pk];
        pos = a.pk_off[h.first_bad_pk];
    } else if (h.walk_err) {
        err = h.walk_err;
        pos = h.walk_err_pos;
    }
    h.error = err;
    c[4] = err;
    c[5] = pos;
    c[3] = 0;
    if (err) {
        c[0] = c[1] = c[2] = 0;
        atomicOr(a.status, RTA_DEV_BAD_STREAM);
        return;
    }
    const unsigned long long last = n > 0 ? a.pk_scan[n - 1] : 0ull;
    c[0] = n;
    c[1] = int64_t(last >> 32);
    c[2] = int64_t(last & 0xFFFFFFFFull);
    if (a.img_seg) a.img_seg[c[1]] = int32_t(n);
    if (a.evt_off) a.evt_off[c[2]] = int32_t(c[1]);
}

// The directory (nothing on a fault).
__global__ void __launch_bounds__(256) k_pkt_emit(const IngestArgs a) {
    if (a.hdr->error) return;
    const int64_t n = a.hdr->n_pk;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        PktFields f;
        const int64_t pos = a.pk_off[k];
        pkt_check(a.stream, pos, a.n_bytes, a.arr, f);
        rta_segment_t sg;
        sg.offset = pos + RTA_PKT_HEADER_BYTES;
        sg.first_pixel = f.first;
        sg.n_pixels = f.n;
        a.seg[k] = sg;
        const unsigned long long incl = a.pk_scan[k];
        const unsigned long long prev = k > 0 ? a.pk_scan[k - 1] : 0ull;
        const int64_t img = int64_t(incl >> 32) - 1, evt = int64_t(incl & 0xFFFFFFFFull) - 1;
        if ((incl >> 32) != (prev >> 32)) {
            a.img_seg[img] = int32_t(k);
            a.img_tel[img] = f.apid;
            atomicAdd(reinterpret_cast<unsigned long long*>(a.counts + 3), (unsigned long long)(f.P) * f.S);
        }
        if ((incl & 0xFFFFFFFFull) != (prev & 0xFFFFFFFFull)) {
            a.evt_off[evt] = int32_t(img);
            a.evt_number[evt] = f.event;
            if (a.evt_time) a.evt_time[evt] = int64_t(f.sec) * 1000000000 + (int64_t(f.fine) * 1000000000) / 65536;
        }
    }
}

// ---------------------------------------------------------------- the image kernel's per-image records
// One thread per image of an ingested stream: the directory checked once (a
// known telescope; segments that tile the camera's pixels in order, 16-byte
// aligned, inside the stream) and packed for the producer.
__global__ void __launch_bounds__(256) k_stream_meta(const ChainArgs a, StreamImg* out, int64_t max_img) {
    const int64_t n = a.n_img_dev ? (*a.n_img_dev < max_img ? *a.n_img_dev : max_img) : max_img;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        StreamImg m = {};
        const int tel = a.img_tel[i];
        bool ok = tel >= 0 && tel < a.arr.n_tel;
        if (ok) {
            m.cam = a.arr.tel_cam[tel];
            const DevCam C = a.arr.cams[m.cam];
            m.P = C.P;
            m.S = C.S;
            m.row = a.arr.tel_row[tel];
        }
        const int seg0 = a.img_seg[i], seg1 = a.img_seg[i + 1];
        ok = ok && seg0 >= 0 && seg1 > seg0 && seg1 <= a.n_seg;
        int next = 0;
        for (int k = seg0; ok && k < seg1; ++k) {
            const rta_segment_t sg = a.seg[k];
            ok = sg.first_pixel == next && sg.n_pixels > 0 && (sg.offset & 15) == 0 &&
                 ((int64_t(sg.n_pixels) * m.S) & 7) == 0 && sg.offset >= 0 &&
                 sg.offset + int64_t(sg.n_pixels) * m.S * 2 <= 2 * a.n_wave;
            if (k - seg0 < STREAM_INLINE_SEGS) {
                m.first[k - seg0] = sg.first_pixel;
                m.n[k - seg0] = sg.n_pixels;
                m.off[k - seg0] = sg.offset;
            }
            next += sg.n_pixels;
        }
        m.ok = ok && next == m.P;
        m.seg0 = seg0;
        m.nseg = ok ? seg1 - seg0 : 0;
        out[i] = m;
    }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_stream_meta(const ChainArgs& a, StreamImg* out, int64_t max_img, int n_sm, cudaStream_t s) {
    const int g = int(std::min<int64_t>((max_img + 255) / 256, int64_t(n_sm) * 8));
    k_stream_meta<<<g > 0 ? g : 1, 256, 0, s>>>(a, out, max_img);
    return cudaGetLastError();
}

int64_t ingest_chunks(int64_t n_bytes) { return (n_bytes + ING_CHUNK - 1) / ING_CHUNK; }

cudaError_t launch_ingest(const IngestArgs& a, int verify_crc, int n_sm, cudaStream_t s) {
    const int64_t nc = a.n_chunks;
    const int64_t max_pk = a.seg_cap + 1;
    const int64_t n_blk = (max_pk + 1023) / 1024;
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.hdr, 0, sizeof(IngHdr), s)) != cudaSuccess) return e;
    k_ingest_init<<<1, 1, 0, s>>>(a);
    k_frame_scan<<<unsigned(nc), ING_SCAN_THREADS, 0, s>>>(a);
    k_frame_join<<<1, 1024, 0, s>>>(a);
    k_frame_list<<<unsigned(nc), 32, 0, s>>>(a);
    const int g = int(std::min<int64_t>((max_pk + 255) / 256, int64_t(n_sm) * 8));
    k_pkt_check<<<g, 256, 0, s>>>(a);
    if (verify_crc) {
        // the dynamic shared-memory opt-in is per device
        static bool attr_set[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !attr_set[dev]) {
            if ((e = cudaFuncSetAttribute(k_pkt_crc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(CRC_SMEM_BYTES))) !=
                cudaSuccess)
                return e;
            if (dev >= 0 && dev < 64) attr_set[dev] = true;
        }
        const int64_t wpb = CRC_THREADS / 32;
        k_pkt_crc<<<int(std::min<int64_t>((max_pk + wpb - 1) / wpb, int64_t(n_sm))), CRC_THREADS, CRC_SMEM_BYTES, s>>>(a);
    }
    k_pkt_scan_local<<<unsigned(n_blk), 1024, 0, s>>>(a);
    k_pkt_scan_blocks<<<1, 1024, 0, s>>>(a, n_blk);
    k_pkt_final<<<unsigned(n_blk), 1024, 0, s>>>(a);
    k_ingest_verdict<<<1, 1, 0, s>>>(a);
    k_pkt_emit<<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rta
