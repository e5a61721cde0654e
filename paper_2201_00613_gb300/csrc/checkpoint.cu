// checkpoint.cu -- save and restore a compact state with its step count.
//
// Host code only (no CUDA calls): the caller copies the state between the
// device and a host buffer.  A checkpoint file is, in little-endian order, a
// 64-byte header (magic "SQZSTATE", format version, header size, s, k, r,
// the number of dimensions (2), the step count, the state size k^r, the
// FNV-1a 64-bit hash of the state and the FNV-1a 64-bit hash of the header
// (this word read as 0) followed by the padded offsets), the 2k offset bytes
// padded with zeros to a multiple of 8, and the k^r state bytes in compact
// order.  FNV-1a changes its hash for any single changed byte, so one
// damaged byte anywhere in the file is caught.  Files are written under a
// temporary name and renamed into place, so a reader sees either the old file
// or the complete new one.
#include <errno.h>
#include <fcntl.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include "squeeze_internal.cuh"

namespace {

constexpr char kMagic[8] = {'S', 'Q', 'Z', 'S', 'T', 'A', 'T', 'E'};
constexpr uint32_t kVersion = 1;

struct Header {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;    // this header plus the padded offsets
  uint32_t s, k, r, dims;
  uint64_t step;
  uint64_t state_bytes;
  uint64_t checksum;        // FNV-1a 64 of the state bytes
  uint64_t header_hash;     // FNV-1a 64 of this header (this word as 0) and the padded offsets
};
static_assert(sizeof(Header) == 64, "checkpoint header layout");

// FNV-1a, 64-bit (Fowler, Noll, Vo): per byte, xor it in, then multiply by
// the FNV prime 2^40 + 2^8 + 0xb3, starting from the offset basis.
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull;
uint64_t fnv1a64(const uint8_t *p, uint64_t n, uint64_t h = kFnvBasis) {
  for (uint64_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

uint64_t header_hash_of(Header hd, const uint8_t *off, uint32_t off_bytes) {
  hd.header_hash = 0;
  return fnv1a64(off, off_bytes, fnv1a64(reinterpret_cast<const uint8_t *>(&hd), sizeof(hd)));
}

uint32_t padded_offsets(uint32_t k) { return (2 * k + 7) / 8 * 8; }

int io_fail(const char *what, const char *path) {
  char text[256];
  const char *why = errno ? strerror(errno) : "bad contents";
  snprintf(text, sizeof(text), "%s %.160s: %.60s", what, path, why);
  sq_set_error_text(text);
  return SQUEEZE_ERR_IO;
}

bool write_all(FILE *fp, const void *p, uint64_t n) {
  const uint8_t *b = static_cast<const uint8_t *>(p);
  while (n) {
    const size_t chunk = n > (1u << 30) ? (1u << 30) : (size_t)n;
    if (fwrite(b, 1, chunk, fp) != chunk) return false;
    b += chunk;
    n -= chunk;
  }
  return true;
}

bool read_all(FILE *fp, void *p, uint64_t n) {
  uint8_t *b = static_cast<uint8_t *>(p);
  while (n) {
    const size_t chunk = n > (1u << 30) ? (1u << 30) : (size_t)n;
    if (fread(b, 1, chunk, fp) != chunk) return false;
    b += chunk;
    n -= chunk;
  }
  return true;
}

}  // namespace

extern "C" {

int squeeze_checkpoint_write(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                             uint64_t step, const uint8_t *h_state, const char *path) {
  sq::FracDev f;
  const int rc = sq_fill_fractal(s, k, offsets, r, f);
  if (rc) return rc;
  if (!h_state || !path || !*path) return SQUEEZE_ERR_INVALID_ARG;
  Header hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, sizeof(kMagic));
  hd.version = kVersion;
  hd.header_bytes = (uint32_t)sizeof(Header) + padded_offsets(k);
  hd.s = s;
  hd.k = k;
  hd.r = r;
  hd.dims = 2;
  hd.step = step;
  hd.state_bytes = f.cells;
  hd.checksum = fnv1a64(h_state, f.cells);
  uint8_t off[2 * 256 + 8];
  memset(off, 0, sizeof(off));
  memcpy(off, offsets, 2 * k);
  hd.header_hash = header_hash_of(hd, off, padded_offsets(k));

  char tmp[4096];
  if (snprintf(tmp, sizeof(tmp), "%s.tmp%ld", path, (long)getpid()) >= (int)sizeof(tmp))
    return SQUEEZE_ERR_INVALID_ARG;
  errno = 0;
  FILE *fp = fopen(tmp, "wb");
  if (!fp) return io_fail("cannot create", tmp);
  bool ok = write_all(fp, &hd, sizeof(hd)) && write_all(fp, off, padded_offsets(k)) &&
            write_all(fp, h_state, f.cells);
  ok = (fflush(fp) == 0) && ok;
  // The data reach the disk before the rename makes them the checkpoint, so
  // a crash cannot leave `path` naming a truncated file.
  ok = (fsync(fileno(fp)) == 0) && ok;
  ok = (fclose(fp) == 0) && ok;
  if (!ok) {
    const int e = errno;
    remove(tmp);
    errno = e;
    return io_fail("cannot write", tmp);
  }
  if (rename(tmp, path) != 0) {
    const int e = errno;
    remove(tmp);
    errno = e;
    return io_fail("cannot rename to", path);
  }
  // Make the rename itself durable: sync the directory that holds the entry.
  char dir[4096];
  snprintf(dir, sizeof(dir), "%s", path);
  char *slash = strrchr(dir, '/');
  if (!slash) snprintf(dir, sizeof(dir), ".");
  else if (slash == dir) dir[1] = 0;
  else *slash = 0;
  const int dfd = open(dir, O_RDONLY | O_DIRECTORY);
  if (dfd >= 0) {
    fsync(dfd);   // best effort: some file systems refuse fsync on a directory
    close(dfd);
  }
  return SQUEEZE_OK;
}

int squeeze_checkpoint_read(uint32_t s, uint32_t k, const uint8_t *offsets, uint32_t r,
                            uint64_t *step, uint8_t *h_state, const char *path) {
  sq::FracDev f;
  const int rc = sq_fill_fractal(s, k, offsets, r, f);
  if (rc) return rc;
  if (!step || !h_state || !path) return SQUEEZE_ERR_INVALID_ARG;
  errno = 0;
  FILE *fp = fopen(path, "rb");
  if (!fp) return io_fail("cannot open", path);
  Header hd;
  uint8_t off[2 * 256 + 8];
  errno = 0;
  bool ok = read_all(fp, &hd, sizeof(hd)) && memcmp(hd.magic, kMagic, sizeof(kMagic)) == 0 &&
            hd.version == kVersion && hd.header_bytes == sizeof(Header) + padded_offsets(hd.k) &&
            hd.dims == 2 && hd.k >= 1 && hd.k <= 256;
  ok = ok && read_all(fp, off, padded_offsets(hd.k));
  if (!ok) {
    fclose(fp);
    return io_fail("not a checkpoint:", path);
  }
  if (header_hash_of(hd, off, padded_offsets(hd.k)) != hd.header_hash) {
    fclose(fp);
    errno = 0;
    return io_fail("damaged checkpoint header:", path);
  }
  // a valid file of another fractal or level is the caller's mistake, not damage
  if (hd.s != s || hd.k != k || hd.r != r || memcmp(off, offsets, 2 * k) != 0 ||
      hd.state_bytes != f.cells) {
    fclose(fp);
    sq_set_error_text("checkpoint holds another fractal or level");
    return SQUEEZE_ERR_INVALID_ARG;
  }
  errno = 0;
  ok = read_all(fp, h_state, f.cells);
  uint8_t extra;
  ok = ok && fread(&extra, 1, 1, fp) == 0 && feof(fp);   // nothing after the state
  fclose(fp);
  if (!ok || fnv1a64(h_state, f.cells) != hd.checksum) return io_fail("damaged checkpoint", path);
  *step = hd.step;
  return SQUEEZE_OK;
}

}  // extern "C"
