// Disk-cache entries of the specialised kernels (tami_jit.cpp): an entry written for one
// compilation identity reads back intact; a foreign identity, and every kind of damage to the file
// (a flipped byte anywhere, truncation, trailing bytes, a wrong magic word or length field), is
// refused before anything would reach the driver; directories are created; an unwritable path
// fails cleanly and leaves no temporary file.  The cubin here is arbitrary bytes and is never
// loaded.  Built and run by tests/test_jit_cache_cpu.py; needs no GPU.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <dirent.h>

#include "tami_internal.h"

using namespace tami;

static int failures = 0;

static void expect(bool ok, bool want, const char* what) {
  if (ok != want) {
    std::printf("FAIL %s\n", what);
    ++failures;
  } else {
    std::printf("%s %s\n", want ? "accepted" : "refused", what);
  }
}

static std::vector<char> slurp(const std::string& p) {
  std::vector<char> b;
  FILE* f = std::fopen(p.c_str(), "rb");
  if (!f) return b;
  int c;
  while ((c = std::fgetc(f)) != EOF) b.push_back((char)c);
  std::fclose(f);
  return b;
}

static void spit(const std::string& p, const std::vector<char>& b) {
  FILE* f = std::fopen(p.c_str(), "wb");
  if (b.size()) std::fwrite(b.data(), 1, b.size(), f);
  std::fclose(f);
}

static int count_entries(const std::string& dir) {
  int n = 0;
  if (DIR* d = opendir(dir.c_str())) {
    while (dirent* e = readdir(d))
      if (e->d_name[0] != '.') ++n;
    closedir(d);
  }
  return n;
}

int main(int argc, char** argv) {
  if (argc < 2) { std::printf("usage: jit_cache_cases <scratch dir>\n"); return 2; }
  const std::string dir = std::string(argv[1]) + "/a/b";
  const std::string path = dir + "/entry.tjc";
  const std::string ident = "nvrtc 13.0\n-arch=sm_103a \nheader text\nsource text";
  std::vector<char> cubin(5000);
  for (size_t i = 0; i < cubin.size(); ++i) cubin[i] = (char)(i * 131 + 7);

  expect(jit_cache_write(path, ident, cubin), true, "write into directories it creates");
  expect(count_entries(dir) == 1, true, "no temporary file left beside the entry");
  std::vector<char> got;
  const bool rd = jit_cache_read(path, ident, &got);
  expect(rd && got == cubin, true, "read back with its identity");

  std::vector<char> sink;
  expect(jit_cache_read(path, ident + "x", &sink), false, "longer identity");
  std::string same_len = ident;
  same_len[same_len.size() - 3] ^= 1;
  expect(jit_cache_read(path, same_len, &sink), false, "identity differing in one byte");
  expect(jit_cache_read(dir + "/missing.tjc", ident, &sink), false, "missing file");

  const std::vector<char> good = slurp(path);
  const size_t at_cubin = 8 + 8 + ident.size() + 8;
  struct Damage { const char* what; size_t pos; };
  const Damage flips[] = {{"flipped magic byte", 3},
                          {"flipped identity-length byte", 8},
                          {"flipped identity byte", 16 + 5},
                          {"flipped cubin-length byte", 8 + 8 + ident.size()},
                          {"flipped first cubin byte", at_cubin},
                          {"flipped middle cubin byte", at_cubin + 2500},
                          {"flipped last cubin byte", at_cubin + cubin.size() - 1},
                          {"flipped checksum byte", good.size() - 1}};
  for (const Damage& d : flips) {
    std::vector<char> b = good;
    b[d.pos] ^= 0x20;
    spit(path, b);
    expect(jit_cache_read(path, ident, &sink), false, d.what);
  }
  {
    std::vector<char> b(good.begin(), good.end() - 1);
    spit(path, b);
    expect(jit_cache_read(path, ident, &sink), false, "truncated by one byte");
    b.assign(good.begin(), good.begin() + at_cubin + 100);
    spit(path, b);
    expect(jit_cache_read(path, ident, &sink), false, "truncated inside the cubin");
    b = good;
    b.push_back(0);
    spit(path, b);
    expect(jit_cache_read(path, ident, &sink), false, "one trailing byte");
    spit(path, std::vector<char>());
    expect(jit_cache_read(path, ident, &sink), false, "empty file");
  }
  // an unwritable target: a path below a regular file
  expect(jit_cache_write(path + "/below/x.tjc", ident, cubin), false, "write below a regular file");
  // rewrite over the damaged entry, then read it again
  expect(jit_cache_write(path, ident, cubin), true, "rewrite over a damaged entry");
  got.clear();
  expect(jit_cache_read(path, ident, &got) && got == cubin, true, "read after the rewrite");
  expect(count_entries(dir) == 1, true, "still one file after the rewrite");
  std::printf("%d failures\n", failures);
  return failures ? 1 : 0;
}
