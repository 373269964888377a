"""GB300-native RTCUR hot path: C-ABI library ``librtcur.so`` plus a thin ctypes binding."""
