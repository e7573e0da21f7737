// File front end (Abstract: the pipeline reads genomes from FASTA files and packs them into 2-bit
// batches).  A FASTA or FASTQ file is read into page-locked host memory by parallel reads of
// disjoint ranges, then parsed and packed on the device by ah_fasta_pack / ah_fastq_pack, whose
// copies from page-locked memory run at the link's full rate.
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cerrno>
#include <cstring>
#include <thread>
#include <vector>

#include "ah_internal.h"

namespace ah {
namespace {

// read the whole file into page-locked memory; *buf is the caller's to cudaFreeHost
ah_status read_file_pinned(ah_ctx* ctx, const char* path, char** buf, uint64_t* n_bytes) {
  *buf = nullptr;
  *n_bytes = 0;
  const int fd = open(path, O_RDONLY);
  if (fd < 0) return fail(ctx, AH_EINVAL, "cannot open %s: %s", path, strerror(errno));
  struct stat st;
  if (fstat(fd, &st) != 0 || !S_ISREG(st.st_mode)) {
    close(fd);
    return fail(ctx, AH_EINVAL, "%s is not a regular file", path);
  }
  const uint64_t size = (uint64_t)st.st_size;
  if (cudaMallocHost((void**)buf, std::max<uint64_t>(1, size)) != cudaSuccess) {
    close(fd);
    *buf = nullptr;
    return fail(ctx, AH_ENOMEM, "page-locked buffer of %llu bytes for %s failed", (unsigned long long)size, path);
  }
  // disjoint ranges of 64 MiB read by up to 8 threads
  constexpr uint64_t kPiece = 64ull << 20;
  const uint64_t pieces = (size + kPiece - 1) / kPiece;
  const unsigned n_threads = (unsigned)std::min<uint64_t>(pieces, std::max(1u, std::min(8u, std::thread::hardware_concurrency())));
  std::atomic<uint64_t> next{0};
  std::atomic<int> bad{0};
  auto reader = [&]() {
    for (uint64_t k; (k = next.fetch_add(1)) < pieces && !bad.load();) {
      uint64_t off = k * kPiece;
      const uint64_t end = std::min(size, off + kPiece);
      while (off < end) {
        const ssize_t r = pread(fd, *buf + off, end - off, (off_t)off);
        if (r < 0 && errno == EINTR) continue;
        if (r <= 0) {
          bad.store(r < 0 ? errno : EIO);
          return;
        }
        off += (uint64_t)r;
      }
    }
  };
  std::vector<std::thread> ts;
  for (unsigned t = 1; t < n_threads; ++t) ts.emplace_back(reader);
  reader();
  for (auto& t : ts) t.join();
  close(fd);
  if (bad.load()) {
    cudaFreeHost(*buf);
    *buf = nullptr;
    return fail(ctx, AH_EINVAL, "reading %s failed: %s", path, strerror(bad.load()));
  }
  *n_bytes = size;
  return AH_OK;
}

}  // namespace
}  // namespace ah

using namespace ah;

extern "C" {

ah_status ah_fasta_pack_file(ah_ctx* ctx, const char* path, const uint32_t* genome_ids, ah_batch** batch_out,
                             ah_fasta** names_out) {
  if (!ctx || !path || !batch_out) return fail(ctx, AH_EINVAL, "ah_fasta_pack_file: NULL argument");
  cudaSetDevice(ctx->device);
  char* text = nullptr;
  uint64_t n = 0;
  ah_status st = read_file_pinned(ctx, path, &text, &n);
  if (st) return st;
  st = ah_fasta_pack(ctx, text, n, genome_ids, batch_out, names_out);
  cudaFreeHost(text);
  return st;
}

ah_status ah_fastq_pack_file(ah_ctx* ctx, const char* path, const uint32_t* genome_ids, ah_batch** batch_out,
                             ah_quals** quals_out, ah_fasta** names_out) {
  if (!ctx || !path || !batch_out || !quals_out) return fail(ctx, AH_EINVAL, "ah_fastq_pack_file: NULL argument");
  cudaSetDevice(ctx->device);
  char* text = nullptr;
  uint64_t n = 0;
  ah_status st = read_file_pinned(ctx, path, &text, &n);
  if (st) return st;
  st = ah_fastq_pack(ctx, text, n, genome_ids, batch_out, quals_out, names_out);
  cudaFreeHost(text);
  return st;
}

}  // extern "C"
