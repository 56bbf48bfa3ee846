/*
 * pivco.h -- C ABI of the GB300 (sm_103a) PivCo-Huffman library.
 *
 * PivCo-Huffman (pivot-coded Huffman) stores each block of 8-bit symbols as a
 * length-limited canonical Huffman code whose bits are "pivoted": every
 * internal node of the code tree owns one bitmap holding, in block order, the
 * next code bit of every symbol whose code passes through that node
 * (paper Sec. 2, Fig. 2-3).  Decoding rebuilds the block bottom-up by merging
 * children's symbol sequences through the node bitmaps (Sec. 3); skewed node
 * bitmaps can be ANS-coded selectively (Sec. 5.2).  The calls below follow the
 * paper's problem statement: histogram -> length-limited code lengths ->
 * tree / pivot layout -> encode blocks -> decode blocks (Sec. 4, App. D).
 *
 * Conventions for every entry point
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  Pointers named "host" are host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued asynchronously on it; nothing here
 *     synchronises unless the comment says "synchronous".
 *   - The device-buffer calls allocate no device memory: scratch space is a
 *     caller-provided workspace sized by a query call (or, for
 *     pivco_decode_blocks_static, an array the library's module holds).  The
 *     exception is the host-buffer codec (pivco_host_codec_*), which owns
 *     device buffers for its pieces: pivco_host_codec_create allocates them
 *     and the first pivco_host_decompress allocates its decode workspaces.
 *   - Blocks are described by `blk_off[nblk + 1]` (device, uint64): block b is
 *     bytes [blk_off[b], blk_off[b+1]) of a flat buffer.
 *   - The return value reports host-side argument errors and launch errors.
 *     Errors found on the device (corrupt input, capacity, a bounded wait that
 *     expired) are written to a caller-provided `int32_t status[nblk]` array
 *     (device) and never trap.
 *
 * Block record (the wire format, App. D adapted to GPU-sized blocks):
 *    0 u32 rec_bytes (multiple of 16)   4 u32 n (symbols)
 *    8 u16 n_int (nodes)  10 u8 kind (0 empty, 1 constant, 2 coded)
 *   11 u8 aux (kind 1: the symbol)  12 "PVC1" (canonical tree) or "PVC2"
 *      (regrouped tree with flat subtrees, Sec. 2.2.3-2.2.4)
 *   kind 2: 16 u8 lens[128] (4-bit code lengths, symbol 2k in the low nibble)
 *          144 u32 n_v[n_int] (symbols through each node, breadth-first order)
 *              u8 marker[n_int] (0 raw; 1..50 | 0x80 XOR: ANS table id;
 *                                0xFF: selected for ANS but stored raw;
 *                                0xF0 + D: flat node of depth D = 2..8)
 *              zero pad to 4, u32 alen[#markers other than 0 and flat]
 *              bodies: raw bodies of the marker-0 and flat nodes
 *                      (ceil(n_v/8) bytes, ceil(n_v*D/8) for a flat node),
 *                      then the bodies of the other nodes; zero pad to 16.
 *   Bitmap bit j is bit (j & 7) of byte j >> 3 (Sec. 2.4.2 bit order).  A
 *   flat node's body holds the D-bit index x of each of its symbols (the
 *   x-th of its 2^D symbols in ascending order), value j at bits
 *   [jD, jD + D), least significant bit first.
 *   The regrouped tree (PVC2): each length class, ascending by symbol, is
 *   cut into groups of the largest power of two left; a group of 2^D is an
 *   item of length l - D; items get canonical codes in (length, first
 *   symbol) order and symbol x of a group the code (item code << D) | x.  A
 *   group of 2^D >= 4 symbols is one flat node; nodes are breadth-first.
 *   An ANS body is u32 nwords[S] for S = ceil(bytes / 16384) segments, then
 *   per segment W = min(32, ceil(seg_bytes / 512)) u32 final rANS states and
 *   nwords u16 renormalisation words.
 */
#ifndef PIVCO_H
#define PIVCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pivco_status;
#define PIVCO_OK 0
#define PIVCO_ERR_INVALID_ARG 1   /* bad argument or parameter */
#define PIVCO_ERR_CAPACITY 2      /* an output or workspace is too small */
#define PIVCO_ERR_CORRUPT 3       /* a record failed validation */
#define PIVCO_ERR_TIMEOUT 4       /* a bounded device wait expired */
#define PIVCO_ERR_CUDA 5          /* a CUDA launch or runtime error */

/* Encoder parameters.  max_len is the code-length limit L (App. D: 11).
 * The ANS fields are the three knobs of the selection rule of Sec. 5.2:
 * a node's bitmap is ANS-coded when it has at least ans_min_bytes bytes (32),
 * its skew max(n0, n1) / n exceeds ans_skew_num / ans_skew_den (5/8 = 0.625),
 * and (depth + fse_H) / (depth + 1) is below ans_ratio_pct / 100 (0.95).
 * flat = 1 codes with the regrouped tree of Sec. 2.2.3-2.2.4 (record tag
 * "PVC2", see the record format above); 0 with the canonical tree ("PVC1").
 * Both kinds of record decode through every decode call. */
typedef struct pivco_params {
    int32_t max_len;
    int32_t ans_enable;
    int32_t ans_min_bytes;
    int32_t ans_skew_num;
    int32_t ans_skew_den;
    int32_t ans_ratio_pct;
    int32_t flat;
} pivco_params;

/* Library version string (host, static storage). */
const char *pivco_version(void);

/* Bytes of the per-block layout record written by pivco_build_layout. */
int32_t pivco_layout_bytes(void);

/* Histogram (Sec. 4: encode-side statistics).  hist[b * 256 + s] (device,
 * uint32) receives the count of byte s in block b.  in: device symbols. */
pivco_status pivco_histogram(const uint8_t *in, const uint64_t *blk_off, int32_t nblk,
                             uint32_t *hist, void *stream);

/* Length-limited code lengths (Sec. 1.2, App. D: limit L = max_len <= 15).
 * Optimal under the limit (package-merge); ties between equal counts are
 * broken by symbol value, so equal-count lower byte values get the longer
 * codes.  lens[b * 256 + s] (device, uint8) is 0 for absent symbols and for
 * blocks with fewer than two distinct symbols.  status[b] (device) gets
 * PIVCO_ERR_INVALID_ARG when 2^max_len is smaller than the alphabet. */
pivco_status pivco_code_lengths(const uint32_t *hist, int32_t nblk, int32_t max_len,
                                uint8_t *lens, int32_t *status, void *stream);

/* Tree / pivot layout (Sec. 2; Sec. 5.2 selection; App. D record layout).
 * From lens and hist builds the canonical codes, the breadth-first node
 * table with per-node counts n_v, the ANS selection of each node, and the
 * record's byte layout.  layout: device buffer of nblk * pivco_layout_bytes()
 * bytes (opaque), 16-byte aligned (else PIVCO_ERR_INVALID_ARG, here and in
 * every call that takes a layout).  rec_bound[b] (device, uint64): the record size with every
 * node stored raw; the final record is never larger.  params: host. */
pivco_status pivco_build_layout(const uint32_t *hist, const uint8_t *lens, int32_t nblk,
                                const pivco_params *params, void *layout, uint64_t *rec_bound,
                                int32_t *status, void *stream);

/* pivco_histogram_chunks, pivco_code_lengths and pivco_build_layout in one
 * launch (one CTA per block; the block's counts and lengths stay on chip
 * between the steps).  Writes exactly what the three calls write: hist,
 * chunk_hist, lens, layout, rec_bound and status (the layout step's). */
pivco_status pivco_plan_blocks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk,
                               const pivco_params *params, uint32_t *hist, uint32_t *chunk_hist,
                               uint8_t *lens, void *layout, uint64_t *rec_bound, int32_t *status,
                               void *stream);

/* Device-wide exclusive scan of n uint64 values (single pass, decoupled
 * look-back): out[0] = 0, out[i+1] = in[0] + ... + in[i] (device arrays,
 * out has n + 1 entries).  Used to place records from their sizes.  ws:
 * device workspace of pivco_scan_workspace_size(n) bytes; status_out: device
 * int32, PIVCO_ERR_TIMEOUT if a look-back wait expired (else untouched). */
size_t pivco_scan_workspace_size(int32_t n);
pivco_status pivco_exclusive_scan(const uint64_t *in, int32_t n, uint64_t *out, void *ws,
                                  size_t ws_bytes, int32_t *status_out, void *stream);

/* Encode blocks (Sec. 4, Table 11: per node, write the bitmap and stably
 * partition the symbols to the non-leaf children).  Writes block b's record at
 * out + out_off[b]; its capacity is out_off[b+1] - out_off[b] and must be at
 * least rec_bound[b], and out + out_off[b] must be 16-byte aligned (else
 * status[b] = PIVCO_ERR_INVALID_ARG and nothing is written).  Nodes selected
 * for ANS are written raw with marker 0xFF; pivco_ans_encode_blocks then codes
 * them.  rec_bytes[b] (device) receives the record size.  status[b] (device). */
pivco_status pivco_encode_blocks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk,
                                 void *layout, uint8_t *out, const uint64_t *out_off,
                                 uint64_t *rec_bytes, int32_t *status, void *stream);

/* The encoder's warp chunks counted in the histogram pass.  Block b of n
 * symbols is cut into nw = min(8, max(1, n / 4096)) contiguous chunks, chunk
 * w starting at floor(n w / nw) rounded down to a multiple of 32 (the split
 * pivco_encode_blocks uses for its warps).  pivco_histogram_chunks writes the
 * block histograms to hist[nblk][256] exactly as pivco_histogram does, and
 * each chunk's histogram to chunk_hist[nblk][8][256] (device; the chunks a
 * block does not have are zeros).  pivco_encode_blocks_chunked is
 * pivco_encode_blocks reading those chunk histograms instead of counting the
 * chunks again; the records are byte-identical.  The encoder codes a block
 * in runs of consecutive chunks whose levels fit its buffers, taking each
 * run's node counts from the summed chunk histograms (a chunk too large for
 * the buffers is coded in parts counted from `in`, and the parts' counts
 * must add up to its histogram).  Chunk histograms that do not describe
 * `in` (another input, or stale) never give a wrong record with an OK
 * status: a block is either refused (status[b] = PIVCO_ERR_INVALID_ARG) or,
 * when the sums it used are right after all, encoded exactly; nothing is
 * written outside each block's record.  A block whose levels do not fit
 * the encoder's buffers is coded chunk by chunk by several CTAs (a work
 * list of (block, chunk) items); each chunk starts at the node cursors its
 * preceding chunks' histograms give.  Both encode calls keep that work list
 * in scratch words at the end of the layout records, so one layout serves
 * one encode call at a time. */
pivco_status pivco_histogram_chunks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk,
                                    uint32_t *hist, uint32_t *chunk_hist, void *stream);
pivco_status pivco_encode_blocks_chunked(const uint8_t *in, const uint64_t *blk_off, int32_t nblk,
                                         void *layout, const uint32_t *chunk_hist, uint8_t *out,
                                         const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status,
                                         void *stream);

/* Selective ANS of encoded records (Sec. 5.2, App. D marker byte): codes the
 * bitmap bytes of every node with marker 0xFF by static-table rANS and keeps
 * the result when it is smaller than the raw bitmap; rewrites the record in
 * place and updates rec_bytes[b].  ws: device workspace of at least
 * out_off[nblk] + 256 * nblk bytes (the encode output size).  status[b]. */
pivco_status pivco_ans_encode_blocks(const void *layout, int32_t nblk, uint8_t *out,
                                     const uint64_t *out_off, uint64_t *rec_bytes, void *ws,
                                     size_t ws_bytes, int32_t *status, void *stream);

/* Decode workspace.  pivco_decode_plan_bytes(nblk) (host, pure) is the size
 * of the plan part of the workspace.  pivco_decode_workspace_size
 * (synchronous) runs the plan for these records in `ws` (device, at least
 * pivco_decode_plan_bytes(nblk) bytes) and returns in *bytes the total
 * workspace pivco_decode_blocks needs (plan plus room for the ANS-decoded
 * bitmaps).  status[b] (device) reports records whose headers are corrupt. */
size_t pivco_decode_plan_bytes(int32_t nblk);
pivco_status pivco_decode_workspace_size(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                         void *ws, size_t ws_bytes, int32_t *status, size_t *bytes,
                                         void *stream);

/* Decode blocks (Sec. 3: bottom-up merge; Sec. 5.2: ANS-coded bitmaps are
 * decoded first).  Record b starts at comp + comp_off[b] (device; at most
 * comp_off[b+1] - comp_off[b] bytes are read).  Symbols go to
 * out + out_off[b]; the capacity out_off[b+1] - out_off[b] must equal the
 * record's n.  ws: device workspace (pivco_decode_workspace_size).  A record
 * must start on a 16-byte boundary (its sizes are multiples of 16, so records
 * placed back to back from an aligned buffer do); one that does not gets
 * PIVCO_ERR_INVALID_ARG and is not read as words.
 * status[b] (device): PIVCO_OK, PIVCO_ERR_CORRUPT, PIVCO_ERR_CAPACITY,
 * PIVCO_ERR_TIMEOUT, PIVCO_ERR_INVALID_ARG. */
pivco_status pivco_decode_blocks(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                 uint8_t *out, const uint64_t *out_off, void *ws, size_t ws_bytes,
                                 int32_t *status, void *stream);

/* pivco_decode_blocks without a caller-supplied workspace.  (The paper has
 * no counterpart: this is an interface convenience of this library.)  It is
 * for callers that cannot allocate device memory at decode time: a plain C
 * caller with no device allocator of its own, or a server whose memory is
 * fully committed to admitted requests, which has nowhere to size a
 * workspace from.  The workspace is instead one library-owned array in
 * device memory of PIVCO_DECODE_STATIC_WS_BYTES (16 MiB), created with the
 * library's module; nothing is allocated per call.
 *   - The first call on each device looks up that array's address (the
 *     module loads then) with that device current, and keeps it for the
 *     life of the process.  Make that first call before any stream capture:
 *     a first call on a stream that is capturing returns
 *     PIVCO_ERR_INVALID_ARG.  The kept address does not survive
 *     cudaDeviceReset; do not call this function after resetting a device
 *     it was called on.
 *   - nblk whose fixed plan part alone (pivco_decode_plan_bytes) exceeds the
 *     array returns PIVCO_ERR_CAPACITY without launching anything.  Blocks
 *     whose ANS scratch or rank directories do not fit in what remains get
 *     status[b] = PIVCO_ERR_CAPACITY (the others decode normally).
 *   - The counters and look-back states that must start at zero are cleared
 *     by the call itself, on `stream`, before its first use of them.
 *   - There is one array per device: calls whose GPU work overlaps (other
 *     streams, other host threads) race on it and give undefined results.
 *     Issue them on one stream, or wait for the previous one.
 * Other arguments, outputs and statuses as pivco_decode_blocks. */
#define PIVCO_DECODE_STATIC_WS_BYTES (16u << 20)
pivco_status pivco_decode_blocks_static(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                        uint8_t *out, const uint64_t *out_off, int32_t *status,
                                        void *stream);

/* ---- Serving (a device-resident request loop; the paper has no serving system) ----
 * A decompression server: a device-resident request loop (one persistent
 * kernel that takes the work items of the batched decode, request after
 * request) fed by a host scheduler thread that admits requests by a device
 * memory budget.  Continuous batching: a request submitted while others run
 * is admitted as soon as budget, arena space and a ring entry are free, and
 * its items run on the device beside those of the requests already there.
 * No request changes what another decodes: each result is the bytes that
 * pivco_decode_blocks gives for it alone.
 *
 * arena: caller-owned device memory (256-byte aligned) the server lives in:
 * a control block and a 4096-entry request ring, then per admitted request
 * its records, offsets, statuses, decode workspace and output.  Nothing is
 * allocated on the device.  Host side the server allocates pinned mapped
 * flags, staging and three non-blocking streams, and runs one thread.
 *
 * pivco_server_submit: `comp` (host, pinned recommended) holds nblk records,
 * record b at comp + comp_off[b]; `out` (host, pinned recommended) receives
 * block b at out + out_off[b]; both must stay valid until the request is
 * done.  comp_off / out_off (host, nblk + 1 entries) are copied at submit.
 * *id receives the request id (ids increase by one per submit).  A request
 * whose device footprint (records + output + offsets + workspace bound)
 * exceeds the budget returns PIVCO_ERR_CAPACITY.
 * pivco_server_poll: *state = 0 unknown, 1 pending (not admitted), 2 admitted,
 * 3 done; for done requests *status = the first non-OK block status (else
 * PIVCO_OK) and *latency_ms = submit to result-in-host-memory.
 * pivco_server_drain waits (at most timeout_ms) until every submitted
 * request is done: PIVCO_ERR_TIMEOUT if not.  pivco_server_forget drops a
 * done request's record.  Device loop waits are bounded; an expired one ends
 * as PIVCO_ERR_TIMEOUT in the request's status. */
typedef struct pivco_server pivco_server;
typedef struct pivco_server_config {
    uint64_t budget_bytes;   /* admission budget (0: the whole arena after its control part) */
    int32_t idle_us;         /* the device loop leaves after this long with nothing to do (default 200) */
    int32_t epoch_us;        /* lifetime of one loop launch before a fresh one takes over (default 4000) */
} pivco_server_config;
pivco_status pivco_server_create(void *arena, size_t arena_bytes, const pivco_server_config *cfg,
                                 pivco_server **srv);
pivco_status pivco_server_submit(pivco_server *srv, const uint8_t *comp, const uint64_t *comp_off,
                                 int32_t nblk, const uint64_t *out_off, uint8_t *out, uint64_t *id);
pivco_status pivco_server_poll(pivco_server *srv, uint64_t id, int32_t *state, int32_t *status,
                               double *latency_ms);
pivco_status pivco_server_drain(pivco_server *srv, int32_t timeout_ms);
pivco_status pivco_server_forget(pivco_server *srv, uint64_t id);
pivco_status pivco_server_destroy(pivco_server *srv);

/* The three steps of pivco_decode_blocks, callable one by one (same
 * arguments and workspace; call them in this order on one stream):
 *   pivco_decode_plan   parses every record header, checks its layout and
 *                       places the ANS work in `ws` (single-pass scan with
 *                       decoupled look-back over the blocks); sets status[b];
 *   pivco_decode_ans    rANS-decodes every ANS-coded node bitmap into the
 *                       workspace (Sec. 5.2), one warp per 16 KiB segment;
 *   pivco_decode_merge  rebuilds the symbols bottom-up (Sec. 3) through
 *                       per-chunk rank directories, one CTA per block. */
pivco_status pivco_decode_plan(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                               size_t ws_bytes, int32_t *status, void *stream);
pivco_status pivco_decode_ans(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                              size_t ws_bytes, int32_t *status, void *stream);
pivco_status pivco_decode_merge(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                uint8_t *out, const uint64_t *out_off, void *ws, size_t ws_bytes,
                                int32_t *status, void *stream);

/* Random access (Sec. 2.1's top-down traversal, answered per position the
 * way a wavelet tree answers access, Sec. 7.2): the symbol at position
 * qpos[i] of block qblk[i] (device arrays of nq uint32), by a walk from the
 * root in which the position's bit at node v picks the child and its rank
 * among the positions of that bit (rank directory + popcount) becomes the
 * position at the child.  Gives the bytes pivco_decode_blocks gives, one
 * position at a time, without decoding the rest of the block.
 *   pivco_access_workspace_size (synchronous): as
 *     pivco_decode_workspace_size, for a workspace that holds a rank
 *     directory for every coded block;
 *   pivco_access_prepare: plans the records, decodes the ANS-coded bitmaps
 *     and builds the directories in `ws` (asynchronous; status[b] as for
 *     pivco_decode_blocks);
 *   pivco_access: the queries, any number of times on a prepared `ws` (the
 *     records and `status` must be those of the prepare).  sym[i] (device
 *     uint8) receives the symbol; qstatus[i] (device int32, may be NULL):
 *     PIVCO_OK, PIVCO_ERR_INVALID_ARG (block index or position out of
 *     range, or a workspace not prepared for access), or the block's
 *     non-OK status, or PIVCO_ERR_CORRUPT (the walk left the tree). */
pivco_status pivco_access_workspace_size(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                                         size_t ws_bytes, int32_t *status, size_t *bytes, void *stream);
pivco_status pivco_access_prepare(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                                  size_t ws_bytes, int32_t *status, void *stream);
pivco_status pivco_access(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, const uint32_t *qblk,
                          const uint32_t *qpos, int32_t nq, uint8_t *sym, int32_t *qstatus, const void *ws,
                          size_t ws_bytes, const int32_t *status, void *stream);

/* ---- PivCo-Golomb (App. G): pivoted coding of Golomb codes ----
 * Values are Golomb-coded with parameter 1 (the unary code): value v is v
 * continue bits then one stop bit, stop = 1.  Pivoted, the code is a list of
 * bitmaps instead of a tree: bitmap j holds, in order, the j-th code bit of
 * every value >= j (1 where the value is j, 0 where it is larger), and the
 * decoder merges the list bottom-up with App. G's merge_vec_cst_plus1
 * (cst 0xFF): out_j[i] = B_j[i] ? 0x00 : out_{j+1}[rank0(B_j, i)] + 1.
 * Record of a block (16-byte aligned, like the PivCo-Huffman record):
 *    0 u32 rec_bytes (multiple of 16)   4 u32 n   8 u16 m (largest value + 1;
 *    0 for an empty block)   10 u8 kind = 4   11 u8 0   12 "PVG1"
 *   16 u32 n_j[m] (values >= j; n_0 = n), then the bitmaps B_0 .. B_{m-1} of
 *      ceil(n_j / 8) bytes each, back to back (bit i in byte i >> 3 at bit
 *      i & 7, pad bits 0), zero pad to 16.
 * Blocks hold at most PIVCO_GOLOMB_MAX_BLOCK values (one CTA keeps a block's
 * levels in shared memory); larger ones get status[b] = PIVCO_ERR_INVALID_ARG.
 *   pivco_golomb_plan: rec_size[b] (device uint64) = the exact record size
 *     of block b of `in` (device values, blocks by blk_off); place records by
 *     an exclusive scan of the sizes (pivco_exclusive_scan);
 *   pivco_golomb_encode: block b's record at out + out_off[b] (capacity
 *     out_off[b+1] - out_off[b], else PIVCO_ERR_CAPACITY), its size in
 *     rec_bytes[b];
 *   pivco_golomb_decode: block b's values at out + out_off[b] (capacity must
 *     equal the record's n, else PIVCO_ERR_CAPACITY); a record that fails
 *     validation gives PIVCO_ERR_CORRUPT.
 * status[b] (device int32) as for the PivCo-Huffman calls. */
#define PIVCO_GOLOMB_MAX_BLOCK 32768u
pivco_status pivco_golomb_plan(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, uint64_t *rec_size,
                               int32_t *status, void *stream);
pivco_status pivco_golomb_encode(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, uint8_t *out,
                                 const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status, void *stream);
pivco_status pivco_golomb_decode(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                 const uint64_t *out_off, int32_t *status, void *stream);

/* Number of kernels this library has launched in this process (host). */
uint64_t pivco_launch_count(void);

/* Bound of the library's device-side waits (process-wide, host).  Every
 * wait a kernel makes on work of another CTA (the decoupled look-backs of
 * pivco_exclusive_scan and of the decode plan, the batched decode's and the
 * serving loop's waits on earlier queue items) gives up after `ns`
 * nanoseconds of device time.  The blocks concerned then report
 * PIVCO_ERR_TIMEOUT (pivco_exclusive_scan: its status_out) and the kernel
 * returns; no block whose work was abandoned reports PIVCO_OK.  Applies to
 * calls issued after it is set (a server takes it at each submit).  Default
 * 10^9 (1 s).  pivco_get_wait_limit returns the current bound. */
pivco_status pivco_set_wait_limit(uint64_t ns);
uint64_t pivco_get_wait_limit(void);

/* ---- Batching (not in the paper: the GPU scheduling of many blocks) ----
 * pivco_decode_batched decodes the same records as pivco_decode_blocks (same
 * arguments, same workspace size, identical output) with one persistent
 * launch whose work queue is keyed by (block, stage): record plans, first
 * tiles (the only tile of a block that needs no ANS segment and no
 * directory, as soon as its own plan is complete), ANS segments, rank
 * directories, the other tiles.  Each item waits (bounded, by default 1 s)
 * only on items earlier in the queue; an expired wait marks the block
 * PIVCO_ERR_TIMEOUT. */
pivco_status pivco_decode_batched(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                  uint8_t *out, const uint64_t *out_off, void *ws, size_t ws_bytes,
                                  int32_t *status, void *stream);

/* Host-buffer codec: compress and decompress a batch of blocks that lives in
 * host memory, the host<->device copies overlapped with the kernels (no
 * counterpart in the paper: a transport convenience of this library).  The
 * blocks (blk_off: host, nblk + 1 offsets, blk_off[0] = 0) are cut into
 * `segments` pieces of about equal raw size; while one piece is coded, the
 * next is copied in and the previous one out.  All buffers below are host
 * memory; page-locked buffers let the copies run asynchronously.
 *   create: device buffers for every piece (about 2x the raw bytes for
 *     records, 2x for input and output); params as for pivco_build_layout.
 *   comp_capacity: the largest compressed size any input can have.
 *   compress: records of in[] into comp[0 .. comp_cap) back to back (the same
 *     bytes pivco_encode_blocks and pivco_ans_encode_blocks write, each
 *     record in its bound-sized slot), comp_off[nblk + 1] their offsets,
 *     status[nblk] per block.  PIVCO_ERR_CAPACITY if comp_cap is too small.
 *   decompress: blocks of comp[] (records at comp_off[b], 16-byte aligned
 *     relative to comp_off[0]) into out[blk_off[b] ..]; status[nblk] as for
 *     pivco_decode_blocks.  The first call allocates each piece's decode
 *     workspace, sized from the block sizes alone (no record is read on the
 *     host; up to about 3x the piece's raw bytes), and later calls reuse it.
 * One call at a time per codec; each call returns when its output is in
 * host memory. */
typedef struct pivco_host_codec pivco_host_codec;
pivco_status pivco_host_codec_create(const uint64_t *blk_off, int32_t nblk, const pivco_params *params,
                                     int32_t segments, pivco_host_codec **codec);
pivco_status pivco_host_codec_destroy(pivco_host_codec *codec);
uint64_t pivco_host_codec_comp_capacity(const pivco_host_codec *codec);
pivco_status pivco_host_compress(pivco_host_codec *codec, const uint8_t *in, uint8_t *comp, uint64_t comp_cap,
                                 uint64_t *comp_off, int32_t *status);
pivco_status pivco_host_decompress(pivco_host_codec *codec, const uint8_t *comp, const uint64_t *comp_off,
                                   uint8_t *out, int32_t *status);

/* Launch tuning of the decode (process-wide).  None of it changes any output.
 * tile_max: longest root tile in symbols (a multiple of 128, 128..2^20;
 *   the plan also caps a tile so that each of its levels fits the CTA's
 *   level buffer; default 2^20);
 * dir_bits: rank-directory granularity in bits (a multiple of 32, 32..256);
 * ctas_per_sm: persistent CTAs per SM (0 = as many as fit, at most 32). */
typedef struct pivco_tuning {
    int32_t tile_max;
    int32_t dir_bits;
    int32_t ctas_per_sm;
    int32_t reserved;
} pivco_tuning;
pivco_status pivco_get_tuning(pivco_tuning *t);
pivco_status pivco_set_tuning(const pivco_tuning *t);

/* Autotuner (synchronous): times pivco_decode_batched on these records under
 * a grid of tunings (tile_max x dir_bits x ctas_per_sm), `reps` launches each,
 * keeps and returns the fastest (*best_ms = its mean time per launch).  The
 * decoded bytes are the same under every tuning.  A tuning whose workspace
 * need (pivco_decode_workspace_size under that tuning) exceeds ws_bytes, or
 * that leaves any status[b] != PIVCO_OK, is never chosen; if none qualifies
 * the tuning is left unchanged and PIVCO_ERR_CAPACITY is returned.  The
 * workspace need depends on the tuning: after changing it, size the
 * workspace again before decoding. */
pivco_status pivco_autotune_decode(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                   uint8_t *out, const uint64_t *out_off, void *ws, size_t ws_bytes,
                                   int32_t *status, int32_t reps, void *stream, pivco_tuning *best,
                                   float *best_ms);

/* CUDA-graph capture of any sequence of the asynchronous calls above on
 * `stream` (not the legacy stream): pivco_graph_begin, then the calls, then
 * pivco_graph_end returns an instantiated graph; pivco_graph_launch replays it
 * (same pointers, same sizes); pivco_graph_destroy frees it (host). */
typedef struct pivco_graph pivco_graph;
pivco_status pivco_graph_begin(void *stream);
pivco_status pivco_graph_end(void *stream, pivco_graph **graph);
pivco_status pivco_graph_launch(pivco_graph *graph, void *stream);
pivco_status pivco_graph_destroy(pivco_graph *graph);

/* The static ANS tables of this library (host, synchronous): fse_h_q16[50]
 * = expected coded bits per bitmap bit in Q16 for tables t = 50..99
 * (Sec. 5.2 fse_H); class_freq[50 * 9] = frequency (out of 2^15) of one byte
 * with k one-bits under table t.  Either pointer may be NULL. */
pivco_status pivco_ans_tables(int32_t *fse_h_q16, uint32_t *class_freq);

/* Standalone ANS of bitmaps (Sec. 5.2).  Bitmap i is bytes
 * [bm_off[i], bm_off[i+1]) of `bitmaps`, coded with table t = table[i] & 0x7F
 * + 49 after XOR with 0xFF when table[i] & 0x80.  pivco_ans_encode writes
 * body i at bodies + body_off[i] (capacity body_off[i+1] - body_off[i], at
 * least 4 * nseg + 132 * nseg + 2 * bytes) and its size to body_bytes[i];
 * pivco_ans_decode inverts it.  All arrays device.  status[i] (device). */
pivco_status pivco_ans_encode(const uint8_t *bitmaps, const uint64_t *bm_off, const uint8_t *table,
                              int32_t nbm, uint8_t *bodies, const uint64_t *body_off,
                              uint64_t *body_bytes, int32_t *status, void *stream);
pivco_status pivco_ans_decode(const uint8_t *bodies, const uint64_t *body_off, const uint8_t *table,
                              int32_t nbm, uint8_t *bitmaps, const uint64_t *bm_off,
                              int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PIVCO_H */
