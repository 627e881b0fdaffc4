// fftseg_stream_file: the paper's pipeline end to end on one GPU (Sec. III).
// A signal file is cut into segments, each segment is transformed, and the
// results are written to an output file in positional order.  The chunker of
// fftseg_stream does the work; the reader and writer here are pread / pwrite
// loops over the two files, optionally with O_DIRECT so that the page cache
// is bypassed and the phase split (fftseg_stream_phases) shows the storage
// itself, the analog of the paper's I/O versus FFT breakdown (Sec. IV).
#include <errno.h>
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include "plan.h"

namespace fftseg {
namespace {

// O_DIRECT wants offsets, sizes and buffers aligned to the device block; the
// chunker's buffers are page-aligned pinned memory, so segment sizes that are
// multiples of kDirectAlign keep every access aligned.
constexpr int64_t kDirectAlign = 4096;

struct FileCtx {
    int fd = -1;
    bool direct = false;
};

int64_t file_read(void *ctx, int64_t offset, void *dst, int64_t bytes)
{
    const FileCtx *f = static_cast<FileCtx *>(ctx);
    const int fd = f->fd;
    const int64_t want = bytes;
    // a short tail under O_DIRECT: ask for whole blocks (the chunker's buffers
    // are whole multiples of them), return only what was asked for
    if (f->direct && bytes % kDirectAlign) bytes += kDirectAlign - bytes % kDirectAlign;
    int64_t done = 0;
    while (done < bytes) {
        const ssize_t r = pread(fd, static_cast<char *>(dst) + done, (size_t)(bytes - done), (off_t)(offset + done));
        if (r < 0) {
            if (errno == EINTR) continue;
            return -1;
        }
        if (r == 0) break;  // end of the file
        done += r;
    }
    return done < want ? done : want;
}

int file_write(void *ctx, int64_t offset, const void *src, int64_t bytes)
{
    const int fd = static_cast<FileCtx *>(ctx)->fd;
    int64_t done = 0;
    while (done < bytes) {
        const ssize_t r =
            pwrite(fd, static_cast<const char *>(src) + done, (size_t)(bytes - done), (off_t)(offset + done));
        if (r < 0) {
            if (errno == EINTR) continue;
            return -1;
        }
        done += r;
    }
    return 0;
}

// open(2) with O_DIRECT when asked, falling back to buffered I/O where the
// file system refuses it
int open_maybe_direct(const char *path, int flags, bool direct, bool *got_direct)
{
    *got_direct = false;
    if (direct) {
        const int fd = open(path, flags | O_DIRECT, 0644);
        if (fd >= 0) {
            *got_direct = true;
            return fd;
        }
        if (errno != EINVAL) return -1;
    }
    return open(path, flags, 0644);
}

}  // namespace
}  // namespace fftseg

using namespace fftseg;

extern "C" int fftseg_stream_file(fftseg_plan p, const char *in_path, const char *out_path, int64_t start_offset,
                                  int64_t end_offset, int64_t chunk_segments, unsigned file_flags,
                                  int64_t *committed_offset)
{
    const bool direct = (file_flags & FFTSEG_FILE_DIRECT) != 0;
    if (committed_offset) *committed_offset = start_offset;
    if (!p || !in_path || !out_path) return set_error(FFTSEG_E_INVALID, "stream_file: NULL plan or path");
    int64_t seg_in = 0, seg_out = 0;
    segment_bytes(p, &seg_in, &seg_out);
    // frame plans read at frame offsets (multiples of hop), so they use the page cache
    const bool want_direct =
        direct && p->path != PATH_FRAMES && seg_in % kDirectAlign == 0 && seg_out % kDirectAlign == 0;
    FileCtx in, out;
    bool in_direct = false, out_direct = false;
    in.fd = open_maybe_direct(in_path, O_RDONLY, want_direct, &in_direct);
    if (in.fd < 0) return set_error(FFTSEG_E_IO, "stream_file: cannot open %s (errno %d)", in_path, errno);
    struct stat st;
    if (fstat(in.fd, &st) != 0) {
        close(in.fd);
        return set_error(FFTSEG_E_IO, "stream_file: cannot stat %s (errno %d)", in_path, errno);
    }
    if (end_offset < 0) {
        close(in.fd);
        return set_error(FFTSEG_E_INVALID, "stream_file: end_offset < 0");
    }
    const int64_t total = end_offset == 0 || end_offset > (int64_t)st.st_size ? (int64_t)st.st_size : end_offset;
    // a fresh run replaces the output; a resumed run, or one of several ranks
    // writing their parts (FFTSEG_FILE_KEEP), keeps what is there
    const bool trunc = start_offset == 0 && !(file_flags & FFTSEG_FILE_KEEP);
    out.fd = open_maybe_direct(out_path, O_WRONLY | O_CREAT | (trunc ? O_TRUNC : 0), want_direct, &out_direct);
    if (out.fd < 0) {
        close(in.fd);
        return set_error(FFTSEG_E_IO, "stream_file: cannot open %s (errno %d)", out_path, errno);
    }
    in.direct = in_direct;
    out.direct = out_direct;
    int rc = fftseg_stream(p, file_read, &in, file_write, &out, total, start_offset, chunk_segments,
                           committed_offset);
    close(in.fd);
    if (close(out.fd) != 0 && (rc == FFTSEG_OK || rc == FFTSEG_E_PARTIAL))
        rc = set_error(FFTSEG_E_IO, "stream_file: closing %s failed (errno %d)", out_path, errno);
    return rc;
}
