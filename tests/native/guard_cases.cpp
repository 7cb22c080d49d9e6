// The C ABI's exception guard (tami_internal.h, guarded): a body that throws std::bad_alloc returns
// TAMI_ENOMEM, any other exception TAMI_EINVAL, each with a message for tami_last_error; a body that
// returns passes its status through.  Built and run by tests/test_host_harness_cpu.py; needs no GPU.
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <system_error>

#include "tami_internal.h"

int main() {
  int fails = 0;
  auto check = [&](int got, int want, const char* msg_part, const char* what) {
    const char* msg = tami_last_error();
    const bool ok = got == want && (!msg_part || (msg && std::strstr(msg, msg_part)));
    std::printf("%s %s (status %d, message \"%s\")\n", ok ? "ok" : "FAIL", what, got, msg ? msg : "");
    fails += !ok;
  };
  check(tami::guarded([]() -> int { throw std::bad_alloc(); }), TAMI_ENOMEM, "out of host memory", "bad_alloc");
  check(tami::guarded([]() -> int { throw std::system_error(std::make_error_code(std::errc::resource_unavailable_try_again)); }),
        TAMI_EINVAL, "host error", "system_error");
  check(tami::guarded([]() -> int { throw 7; }), TAMI_EINVAL, "host error", "non-standard exception");
  check(tami::guarded([]() -> int { return TAMI_EUNSUPPORTED; }), TAMI_EUNSUPPORTED, nullptr, "status passed through");
  check(tami::guarded([]() -> int { return TAMI_OK; }), TAMI_OK, nullptr, "success passed through");
  std::printf("%d failures\n", fails);
  return fails ? 1 : 0;
}
