// sbf_fastx.cu -- incremental FASTA/FASTQ parser (host code).
//
// Turns FASTX text into the library's read batches (concatenated sequence
// bytes + offsets), one piece per record, without holding a whole file or a
// whole record in memory.  Text may arrive in chunks of any size; a record
// longer than the caller's output buffer is split, and the next piece of the
// record starts with the record's last k-1 bases, so every k-mer of the
// record lies in exactly one piece (no k-mer lost or counted twice).
// Sequence bytes are copied as they are (an N or any other non-ACGT byte is
// invalid for the kernels and breaks k-mers, Sec. IV-F); line breaks, CR and
// blanks inside sequence lines are dropped.
#include <cstring>
#include <new>
#include <vector>

#include "sbf_internal.h"

namespace {

enum State : int {
  kSeek,        // before the first record: skip to a line starting with '>' or '@'
  kHeader,      // inside a '>' or '@' header line
  kFastaSeq,    // FASTA sequence lines, at a line start when line_start is set
  kFastqSeq,    // FASTQ sequence lines (until a line starting with '+')
  kFastqPlus,   // the '+' separator line
  kFastqQual,   // quality bytes (as many as the record has bases)
};

// First '\n' in [p, p + n), or NULL.
inline const uint8_t* line_end(const uint8_t* p, uint64_t n) {
  return static_cast<const uint8_t*>(std::memchr(p, '\n', n));
}

}  // namespace

struct sbf_fastx {
  int k = 31;
  int state = kSeek;
  bool fastq = false;
  bool line_start = true;
  bool open = false;            // a record has started and not ended
  uint64_t next_record = 0;     // index the next record gets
  uint64_t record = 0;          // index of the open record
  uint64_t rec_bases = 0;       // bases of the open record so far (FASTQ quality count)
  uint64_t qual_left = 0;       // quality bytes still to skip
  std::vector<uint8_t> tail;    // the open record's last k-1 bases
};

extern "C" {

int sbf_fastx_create(int k, sbf_fastx** out) {
  sbf::clear_error();
  if (!out) return sbf::fail(SBF_EINVAL, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > 32) return sbf::fail(SBF_EINVAL, "k must be in [1, 32] (got %d)", k);
  sbf_fastx* p = new (std::nothrow) sbf_fastx();
  if (!p) return sbf::fail(SBF_ENOMEM, "host allocation failed");
  p->k = k;
  *out = p;
  return SBF_OK;
}

void sbf_fastx_destroy(sbf_fastx* p) { delete p; }

int sbf_fastx_parse(sbf_fastx* p, const uint8_t* text, uint64_t text_len, int final,
                    uint8_t* seq, uint64_t seq_cap, uint64_t* off, uint64_t* rec,
                    uint64_t pieces_cap, uint64_t* n_pieces, uint64_t* seq_len,
                    uint64_t* consumed) {
  sbf::clear_error();
  if (!p || !seq || !off || !rec || !n_pieces || !seq_len || !consumed || (text_len && !text))
    return sbf::fail(SBF_EINVAL, "NULL argument");
  const uint64_t km1 = (uint64_t)p->k - 1;
  if (seq_cap < 2 * km1 + 64) return sbf::fail(SBF_EINVAL, "seq_cap must be at least 2(k-1) + 64");
  if (pieces_cap < 1) return sbf::fail(SBF_EINVAL, "pieces_cap must be at least 1");

  uint64_t n = 0, pos = 0;
  bool piece = false;  // piece n is open in this batch
  auto open_piece = [&](bool continuing) {
    off[n] = pos;
    rec[n] = p->record;
    piece = true;
    if (continuing) {  // a split record resumes with its last k-1 bases
      std::memcpy(seq + pos, p->tail.data(), p->tail.size());
      pos += p->tail.size();
    }
  };
  auto close_piece = [&]() {
    if (!piece) return;
    ++n;
    off[n] = pos;
    piece = false;
  };
  // a record left open by the previous batch (inside its header or sequence
  // lines) continues in a new piece
  if (p->open && (p->state == kHeader || p->state == kFastaSeq || p->state == kFastqSeq))
    open_piece(true);

  uint64_t i = 0;
  bool full = false;
  while (i < text_len && !full) {
    const uint8_t c = text[i];
    switch (p->state) {
      case kSeek:
        if (p->line_start && (c == '>' || c == '@')) {
          if (n == pieces_cap) { full = true; continue; }
          p->fastq = (c == '@');
          p->record = p->next_record++;
          p->open = true;
          p->rec_bases = 0;
          p->tail.clear();
          p->state = kHeader;
          open_piece(false);
          p->line_start = false;
          ++i;
          break;
        }
        if (c == '\n') {
          p->line_start = true;
          ++i;
        } else {  // skip the rest of the line
          const uint8_t* nl = line_end(text + i, text_len - i);
          p->line_start = nl != nullptr;
          i = nl ? (uint64_t)(nl - text) + 1 : text_len;
        }
        break;
      case kHeader: {
        const uint8_t* nl = line_end(text + i, text_len - i);
        if (nl) {
          p->state = p->fastq ? kFastqSeq : kFastaSeq;
          p->line_start = true;
          i = (uint64_t)(nl - text) + 1;
        } else {
          i = text_len;
        }
        break;
      }
      case kFastaSeq:
      case kFastqSeq: {
        if (p->line_start) {
          const bool ends = p->state == kFastaSeq ? (c == '>' || c == '@') : (c == '+');
          if (ends) {
            if (p->state == kFastqSeq) {  // the record's bases are known: skip the '+' line
              p->state = kFastqPlus;
              p->line_start = false;
              ++i;
              break;
            }
            close_piece();  // a FASTA record ends where the next header starts
            p->open = false;
            p->state = kSeek;
            break;  // kSeek sees the header byte at a line start
          }
        }
        if (c == '\n') {
          p->line_start = true;
          ++i;
          break;
        }
        p->line_start = false;
        // copy the rest of the line (or of the text, or what the output
        // holds), dropping CR and blanks: every sequence byte is above 0x20
        const uint8_t* nl = line_end(text + i, text_len - i);
        uint64_t end = nl ? (uint64_t)(nl - text) : text_len;
        if (end - i > seq_cap - pos) end = i + (seq_cap - pos);
        const uint64_t pos0 = pos;
        for (uint64_t j = i; j < end; ++j) {
          const uint8_t b = text[j];
          seq[pos] = b;
          pos += b > 0x20u;
        }
        p->rec_bases += pos - pos0;
        i = end;
        if (pos == seq_cap && i < text_len && text[i] != '\n') {
          // output full inside a line: split the record here (a byte that
          // would be dropped anyway just waits for the next call)
          const uint64_t piece_len = pos - off[n];
          const uint64_t keep = piece_len < km1 ? piece_len : km1;
          p->tail.assign(seq + pos - keep, seq + pos);
          close_piece();
          full = true;
        }
        break;
      }
      case kFastqPlus:
        if (c == '\n') {
          close_piece();
          p->qual_left = p->rec_bases;
          p->state = kFastqQual;
          p->line_start = true;
          if (p->qual_left == 0) {
            p->open = false;
            p->state = kSeek;
          }
        }
        ++i;
        break;
      case kFastqQual: {
        if (c == '\n' || c == '\r') {
          ++i;
          break;
        }
        // quality bytes up to the line end (CR excluded), at most qual_left
        const uint8_t* nl = line_end(text + i, text_len - i);
        uint64_t end = nl ? (uint64_t)(nl - text) : text_len;
        uint64_t cnt = end - i;
        if (end > i && text[end - 1] == '\r') --cnt;
        if (cnt >= p->qual_left) {
          i += p->qual_left;
          p->qual_left = 0;
          p->open = false;
          p->state = kSeek;
          p->line_start = false;  // the rest of the quality line is skipped by kSeek
        } else {
          p->qual_left -= cnt;
          i = end;
        }
        break;
      }
    }
  }
  if (final && !full && i == text_len) {  // end of input: the open record ends
    close_piece();
    p->open = false;
    p->state = kSeek;
    p->line_start = true;
    p->tail.clear();
  } else if (piece && !full) {
    // the batch ends inside a record's sequence: its next piece resumes with
    // the last k-1 bases
    const uint64_t piece_len = pos - off[n];
    const uint64_t keep = piece_len < km1 ? piece_len : km1;
    p->tail.assign(seq + pos - keep, seq + pos);
    close_piece();
  } else if (piece) {
    close_piece();
  }
  off[n] = pos;
  *n_pieces = n;
  *seq_len = pos;
  *consumed = i;
  return SBF_OK;
}

}  // extern "C"
